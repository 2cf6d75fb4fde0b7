// locator.cu -- learned locator: a 128-256-256-3 MLP that maps the 4x4x4
// neighbourhood of a pierced plaquette to the sub-grid core position inside
// it.  It has no counterpart in the paper; it is trained on positions made by
// the plain localization (Sec. 3.3.3, Eq. 6, localize_impl.cuh), which stays
// both its fallback and the judge of its error.
//
// Encoding: block node (a, b, c), a, b, c in 0..3, is the grid node
// min_corner + (a-1) e_u + (b-1) e_v + (c-1) e_n in the face frame
// (u, v, n) = (x, y, z) / (y, z, x) / (z, x, y) for xy / yz / zx faces; psi is
// conjugated for W = -1 and divided by the RMS of |psi| over the block; the
// input vector is BF16 [((c * 4 + b) * 4 + a) * 2 + {Re, Im}].
//
// Dense layers run on the tensor cores: BF16 operands, FP32 accumulation,
// mma.sync m16n8k16 on 64 x 64 tiles staged in shared memory.  The 256 -> 3
// output layer, the loss, bias sums and Adam run on the FP32 pipes.
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_bf16.h>

#include "localize_impl.cuh"

namespace qtv {

namespace {

constexpr int kIn = 128, kH = 256, kOut = 3;
constexpr size_t kOffW1 = 0, kOffB1 = kOffW1 + (size_t)kH * kIn, kOffW2 = kOffB1 + kH,
                 kOffB2 = kOffW2 + (size_t)kH * kH, kOffW3 = kOffB2 + kH,
                 kOffB3 = kOffW3 + (size_t)kOut * kH, kNumParams = kOffB3 + kOut;
static_assert(kNumParams == QTV_LOCATOR_PARAMS, "parameter count");

__device__ __forceinline__ uint16_t f2bf(float f) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}
__device__ __forceinline__ float bf2f(uint16_t b) {
  return __bfloat162float(__ushort_as_bfloat16(b));
}

// ---------------------------------------------------------------------------
// encoding: four lanes per face, eight faces per warp.  For every orientation
// the 4 x 4 x 4 block is the box [i-1, i+2] x [j-1, j+2] x [k-1, k+2] around
// the face's min corner (i, j, k): lane s of a face's four holds the column
// x = i - 1 + s and walks the 16 (y, z) rows of the box, so each of its 16
// loads reads, with its three partners, 32 contiguous bytes of one grid row.
// The orientation only decides where node (s, dy, dz) of the box lands in the
// input vector: block node (a, b, c) of the frame (u, v, w) is
//   o = 0 (u, v, w) = (x, y, z): (a, b, c) = (s, dy, dz)
//   o = 1 (u, v, w) = (y, z, x): (a, b, c) = (dy, dz, s)
//   o = 2 (u, v, w) = (z, x, y): (a, b, c) = (dz, s, dy)
// and P0 = block node (1, 1, 1) is the min corner itself (s = dy = dz = 1).
// For o = 1 and 2 a lane's words fall in runs of four (16-byte stores); for
// o = 0 the four lanes of a face fill 16 contiguous bytes per store.  Against
// a warp per face (every lane repeating the face's index arithmetic, 347
// warp instructions a face) this runs 0.47 -> 0.20 ms for the 1.39e6 faces
// of the 512^3 bench field; 64 registers (four blocks a multiprocessor) beat
// 78 even with a few bytes spilled.
// ---------------------------------------------------------------------------
constexpr int kEncFacesPerWarp = 8;

// faces f in [f0, min(f0 + m, nn)) with nn = min(n, *n_dev); outputs at row f - f0
__global__ void __launch_bounds__(256, 4) encode_kernel(
    const __grid_constant__ FaceGeo geo, unsigned long long f0, unsigned long long m,
    unsigned long long n, const uint64_t* __restrict__ n_dev, const uint64_t* __restrict__ face_ids,
    const int8_t* __restrict__ winding, uint16_t* __restrict__ xo, uint8_t* __restrict__ oko,
    float* __restrict__ rmso) {
  unsigned long long nn = n;
  if (n_dev) nn = *n_dev < n ? *n_dev : n;
  if (f0 + m < nn) nn = f0 + m;
  const int lane = threadIdx.x & 31, s = lane & 3;
  const int g0 = lane & ~3;  // first lane of this face's four
  const unsigned long long warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long fw = f0 + kEncFacesPerWarp *
                                        (((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
       fw < nn; fw += kEncFacesPerWarp * warps) {
    const unsigned long long f = fw + (unsigned)(lane >> 2);
    const bool act = f < nn;
    const uint64_t id = act ? face_ids[f] : 3ull;  // orientation 3: no face
    const bool conjg = act && winding[f] == -1;
    const GridGeo& G = geo.g[act ? geo_snapshot(geo, f) : 0];
    const float2* __restrict__ psi = G.psi;
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const int o = (int)(id & 3u);
    long long ci, cj, ck;
    split_lin(id >> 2, nx, ny, ci, cj, ck);
    const long long px = ci - 1 + s;
    const bool xin = o != 3 && px >= 0 && px < nx;
    bool inside = xin;
    float2 v[16];
#pragma unroll
    for (int dz = 0; dz < 4; ++dz) {
      const long long pz = ck - 1 + dz;
#pragma unroll
      for (int dy = 0; dy < 4; ++dy) {
        const long long py = cj - 1 + dy;
        const bool in = xin && py >= 0 && py < ny && pz >= 0 && pz < nz;
        inside = inside && in;
        v[4 * dz + dy] = in ? __ldg(psi + (pz * ny + py) * nx + px) : make_float2(0.f, 0.f);
      }
    }
    if (conjg) {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i].y = -v[i].y;
    }
    // rotate by conj(P0)/|P0|, P0 = box node (s, dy, dz) = (1, 1, 1)
    {
      const float p0r = __shfl_sync(0xffffffffu, v[5].x, g0 + 1);
      const float p0i = __shfl_sync(0xffffffffu, v[5].y, g0 + 1);
      const float m0 = sqrtf(p0r * p0r + p0i * p0i);
      if (m0 > 0.f) {
        const float cr = p0r / m0, cim = -p0i / m0;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float re = v[i].x * cr - v[i].y * cim;
          const float im = v[i].x * cim + v[i].y * cr;
          v[i] = make_float2(re, im);
        }
      }
    }
    float s2 = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) s2 += v[i].x * v[i].x + v[i].y * v[i].y;
    s2 += __shfl_xor_sync(0xffffffffu, s2, 1);
    s2 += __shfl_xor_sync(0xffffffffu, s2, 2);
    int all_in = inside ? 1 : 0;
    all_in &= __shfl_xor_sync(0xffffffffu, all_in, 1);
    all_in &= __shfl_xor_sync(0xffffffffu, all_in, 2);
    const float rr = sqrtf(s2 * (1.f / 64.f));
    const bool good = all_in && rr > 0.f && rr <= 3.0e38f;
    const float inv = good ? 1.f / rr : 0.f;
    if (act) {
      uint32_t wd[16];  // BF16 pairs, box order 4 dz + dy
#pragma unroll
      for (int i = 0; i < 16; ++i)
        wd[i] = (uint32_t)f2bf(v[i].x * inv) | ((uint32_t)f2bf(v[i].y * inv) << 16);
      uint32_t* x = reinterpret_cast<uint32_t*>(xo + (f - f0) * kIn);
      if (o == 1) {  // q = 16 s + 4 dz + dy: this lane's 16 words are contiguous
#pragma unroll
        for (int dz = 0; dz < 4; ++dz)
          reinterpret_cast<uint4*>(x)[4 * s + dz] =
              make_uint4(wd[4 * dz], wd[4 * dz + 1], wd[4 * dz + 2], wd[4 * dz + 3]);
      } else if (o == 2) {  // q = 16 dy + 4 s + dz: four contiguous words per dy
#pragma unroll
        for (int dy = 0; dy < 4; ++dy)
          reinterpret_cast<uint4*>(x)[4 * dy + s] =
              make_uint4(wd[dy], wd[4 + dy], wd[8 + dy], wd[12 + dy]);
      } else {  // q = s + 4 dy + 16 dz: the four lanes fill 16 contiguous bytes
#pragma unroll
        for (int i = 0; i < 16; ++i) x[s + 4 * i] = wd[i];
      }
      if (s == 0) {
        oko[f - f0] = good ? 1 : 0;
        rmso[f - f0] = good ? rr : 0.f;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// BF16 GEMM on the tensor cores: C[M x N] = op(A)[M x K] * op(B)[K x N].
//   A: AT ? stored [K][M] : stored [M][K];   B: BT ? stored [K][N] : stored [N][K]
// (B stored [N][K] is the (out, in) weight layout).  N % 64 == 0, K % 32 == 0.
// Epilogues: EPI_STORE_F32 C; EPI_BIAS_RELU_BF16 relu(C + bias) as BF16;
// EPI_RELU_MASK_BF16 C * (mask > 0) as BF16 (backward through a ReLU).
// ---------------------------------------------------------------------------
enum { EPI_STORE_F32 = 0, EPI_BIAS_RELU_BF16 = 1, EPI_RELU_MASK_BF16 = 2 };
constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8;

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <bool AT, bool BT, int EPI>
__global__ void __launch_bounds__(128) gemm_bf16_kernel(int M, int N, int K,
                                                        const uint16_t* __restrict__ A, int lda,
                                                        const uint16_t* __restrict__ B, int ldb,
                                                        void* __restrict__ Cout, int ldc,
                                                        const float* __restrict__ bias,
                                                        const uint16_t* __restrict__ mask) {
  __shared__ __align__(16) uint16_t As[GBM][GBK + GPAD];
  __shared__ __align__(16) uint16_t Bs[GBN][GBK + GPAD];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int g = lane >> 2, tg = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

  for (int k0 = 0; k0 < K; k0 += GBK) {
    // A tile -> As[m][k]
    if (!AT) {
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        const int ch = tid + it * 128;  // 256 chunks of 8 along k
        const int mm = ch >> 2, kk = (ch & 3) * 8;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (m0 + mm < M) v = *reinterpret_cast<const uint4*>(A + (size_t)(m0 + mm) * lda + k0 + kk);
        *reinterpret_cast<uint4*>(&As[mm][kk]) = v;
      }
    } else {
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        const int ch = tid + it * 128;  // 256 chunks of 8 along m
        const int kk = ch >> 3, mm = (ch & 7) * 8;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (m0 + mm < M) v = *reinterpret_cast<const uint4*>(A + (size_t)(k0 + kk) * lda + m0 + mm);
        const uint16_t* e = reinterpret_cast<const uint16_t*>(&v);
#pragma unroll
        for (int q = 0; q < 8; ++q) As[mm + q][kk] = e[q];
      }
    }
    // B tile -> Bs[n][k]
    if (!BT) {
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        const int ch = tid + it * 128;
        const int nn = ch >> 2, kk = (ch & 3) * 8;
        *reinterpret_cast<uint4*>(&Bs[nn][kk]) =
            *reinterpret_cast<const uint4*>(B + (size_t)(n0 + nn) * ldb + k0 + kk);
      }
    } else {
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        const int ch = tid + it * 128;
        const int kk = ch >> 3, nn = (ch & 7) * 8;
        const uint4 v = *reinterpret_cast<const uint4*>(B + (size_t)(k0 + kk) * ldb + n0 + nn);
        const uint16_t* e = reinterpret_cast<const uint16_t*>(&v);
#pragma unroll
        for (int q = 0; q < 8; ++q) Bs[nn + q][kk] = e[q];
      }
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < GBK; ks += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + i * 16 + g;
        af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][ks + tg * 2]);
        af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + tg * 2]);
        af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][ks + tg * 2 + 8]);
        af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + tg * 2 + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + j * 8 + g;
        bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + tg * 2]);
        bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + tg * 2 + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
    }
    __syncthreads();
  }
  // epilogue
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int row = m0 + wm + i * 16 + g + hh * 8;
        const int col = n0 + wn + j * 8 + tg * 2;
        if (row >= M) continue;
        float v0 = acc[i][j][hh * 2], v1 = acc[i][j][hh * 2 + 1];
        if (EPI == EPI_STORE_F32) {
          float* C = reinterpret_cast<float*>(Cout);
          *reinterpret_cast<float2*>(C + (size_t)row * ldc + col) = make_float2(v0, v1);
        } else {
          if (EPI == EPI_BIAS_RELU_BF16) {
            v0 = fmaxf(v0 + bias[col], 0.f);
            v1 = fmaxf(v1 + bias[col + 1], 0.f);
          } else {
            const uint32_t mk = *reinterpret_cast<const uint32_t*>(mask + (size_t)row * ldc + col);
            if (bf2f((uint16_t)(mk & 0xffffu)) <= 0.f) v0 = 0.f;
            if (bf2f((uint16_t)(mk >> 16)) <= 0.f) v1 = 0.f;
          }
          uint16_t* C = reinterpret_cast<uint16_t*>(Cout);
          *reinterpret_cast<uint32_t*>(C + (size_t)row * ldc + col) =
              (uint32_t)f2bf(v0) | ((uint32_t)f2bf(v1) << 16);
        }
      }
}

template <bool AT, bool BT, int EPI>
int gemm(int M, int N, int K, const uint16_t* A, int lda, const uint16_t* B, int ldb, void* C,
         int ldc, const float* bias, const uint16_t* mask, cudaStream_t st) {
  if (M <= 0) return QTV_OK;
  if (N % GBN || K % GBK) return set_error(QTV_ERR_ARG, "gemm: N %% 64 or K %% 32 not zero");
  const dim3 grid(N / GBN, (M + GBM - 1) / GBM);
  gemm_bf16_kernel<AT, BT, EPI><<<grid, 128, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, mask);
  return check_cuda(cudaGetLastError(), "gemm_bf16_kernel launch");
}

// ---------------------------------------------------------------------------
// small FP32 kernels
// ---------------------------------------------------------------------------
// y = A2 W3^T + b3 (one thread per row); optionally loss and dY = 2 (y - t) / B
__global__ void out_layer_kernel(const uint16_t* __restrict__ A2, const float* __restrict__ P,
                                 unsigned long long n, float* __restrict__ y,
                                 const float* __restrict__ t, float* __restrict__ dy,
                                 float* __restrict__ loss) {
  __shared__ float w3[kOut * kH + kOut];
  for (int i = threadIdx.x; i < kOut * kH + kOut; i += blockDim.x) w3[i] = P[kOffW3 + i];
  __syncthreads();
  float lsum = 0.f;
  for (unsigned long long m = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; m < n;
       m += (unsigned long long)gridDim.x * blockDim.x) {
    float o0 = w3[kOut * kH], o1 = w3[kOut * kH + 1], o2 = w3[kOut * kH + 2];
    const uint4* row = reinterpret_cast<const uint4*>(A2 + m * kH);
    for (int c = 0; c < kH / 8; ++c) {
      const uint4 v = row[c];
      const uint16_t* e = reinterpret_cast<const uint16_t*>(&v);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float a = bf2f(e[q]);
        const int k = c * 8 + q;
        o0 = fmaf(a, w3[k], o0);
        o1 = fmaf(a, w3[kH + k], o1);
        o2 = fmaf(a, w3[2 * kH + k], o2);
      }
    }
    if (y) {
      y[3 * m] = o0;
      y[3 * m + 1] = o1;
      y[3 * m + 2] = o2;
    }
    if (t) {
      const float d0 = o0 - t[3 * m], d1 = o1 - t[3 * m + 1], d2 = o2 - t[3 * m + 2];
      lsum += d0 * d0 + d1 * d1 + d2 * d2;
      const float sc = 2.f / (float)n;
      dy[3 * m] = sc * d0;
      dy[3 * m + 1] = sc * d1;
      dy[3 * m + 2] = sc * d2;
    }
  }
  if (t) {  // per-block loss into loss[blockIdx.x] (summed in block order later)
    __shared__ float ws[32];
    for (int d = 16; d; d >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, d);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      float b = 0.f;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) b += ws[i];
      loss[blockIdx.x] = b / (float)n;
    }
  }
}

// dH2[m][k] = (sum_o dY[m][o] W3[o][k]) * (A2[m][k] > 0), BF16
__global__ void out_back_kernel(const float* __restrict__ dy, const float* __restrict__ P,
                                const uint16_t* __restrict__ A2, unsigned long long n,
                                uint16_t* __restrict__ dH2) {
  for (unsigned long long idx = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
       idx < n * kH; idx += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long m = idx / kH;
    const int k = (int)(idx % kH);
    float v = dy[3 * m] * P[kOffW3 + k] + dy[3 * m + 1] * P[kOffW3 + kH + k] +
              dy[3 * m + 2] * P[kOffW3 + 2 * kH + k];
    if (bf2f(A2[idx]) <= 0.f) v = 0.f;
    dH2[idx] = f2bf(v);
  }
}

constexpr int kRowChunk = 64;  // rows per block of the reductions below
constexpr int kSplits = 16;    // most K splits of a weight-gradient GEMM on tcgen05
constexpr int kLossBlocks = 1024;                     // most blocks of the loss
constexpr int kPartW3 = kOut * kH + kOut;             // W3 and b3 partials per chunk

// partial dW3[o][k] = sum_m dY[m][o] A2[m][k] and db3[o] = sum_m dY[m][o] over
// one chunk of rows per block (thread k = 0..kH, k == kH the bias), into
// part[block][kOut kH + kOut] (the layout of W3 and b3 in the parameters)
__global__ void out_wgrad_kernel(const float* __restrict__ dy, const uint16_t* __restrict__ A2,
                                 unsigned long long n, float* __restrict__ part) {
  const int k = threadIdx.x;
  const unsigned long long m0 = (unsigned long long)blockIdx.x * kRowChunk;
  const unsigned long long m1 = m0 + kRowChunk < n ? m0 + kRowChunk : n;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  for (unsigned long long m = m0; m < m1; ++m) {
    const float a = k < kH ? bf2f(A2[m * kH + k]) : 1.f;
    s0 = fmaf(dy[3 * m], a, s0);
    s1 = fmaf(dy[3 * m + 1], a, s1);
    s2 = fmaf(dy[3 * m + 2], a, s2);
  }
  float* out = part + (size_t)blockIdx.x * (kOut * kH + kOut);
  if (k < kH) {
    out[k] = s0;
    out[kH + k] = s1;
    out[2 * kH + k] = s2;
  } else if (k == kH) {
    out[kOut * kH] = s0;
    out[kOut * kH + 1] = s1;
    out[kOut * kH + 2] = s2;
  }
}

// part[block][k] = column sums of a BF16 [n x kH] matrix over one chunk of rows
__global__ void colsum_kernel(const uint16_t* __restrict__ D, unsigned long long n,
                              float* __restrict__ part) {
  const int k = threadIdx.x;
  const unsigned long long m0 = (unsigned long long)blockIdx.x * kRowChunk;
  const unsigned long long m1 = m0 + kRowChunk < n ? m0 + kRowChunk : n;
  float s = 0.f;
  for (unsigned long long m = m0; m < m1; ++m) s += bf2f(D[m * kH + k]);
  part[(size_t)blockIdx.x * kH + k] = s;
}

// out[i] = sum over blocks b = 0, 1, ... of part[b][i], in that order (the
// reductions over the batch give the same result on every run)
__global__ void sum_parts_kernel(const float* __restrict__ part, int nb, int width,
                                 float* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < width; i += gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int b = 0; b < nb; ++b) acc += part[(size_t)b * width + i];
    out[i] = acc;
  }
}

// Adam (Kingma & Ba), bias-corrected; refreshes the BF16 copies of W1, W2
__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ G,
                            float* __restrict__ Mo, float* __restrict__ Vo, int n, float lr,
                            float b1, float b2, float eps, float c1, float c2,
                            uint16_t* __restrict__ w1b, uint16_t* __restrict__ w2b,
                            uint16_t* __restrict__ w2tb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float g = G[i];
    const float m = b1 * Mo[i] + (1.f - b1) * g;
    const float v = b2 * Vo[i] + (1.f - b2) * g * g;
    Mo[i] = m;
    Vo[i] = v;
    const float p = P[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    P[i] = p;
    if (i < (int)kOffB1) {
      w1b[i - kOffW1] = f2bf(p);
    } else if (i >= (int)kOffW2 && i < (int)kOffB2) {
      const int j = i - (int)kOffW2;  // W2[o][k], j = o kH + k
      w2b[j] = f2bf(p);
      w2tb[(j % kH) * kH + j / kH] = f2bf(p);
    }
  }
}

__global__ void refresh_bf16_kernel(const float* __restrict__ P, uint16_t* __restrict__ w1b,
                                    uint16_t* __restrict__ w2b, uint16_t* __restrict__ w2tb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kH * kIn + kH * kH;
       i += gridDim.x * blockDim.x) {
    if (i < kH * kIn) {
      w1b[i] = f2bf(P[kOffW1 + i]);
    } else {
      const int j = i - kH * kIn;
      const uint16_t b = f2bf(P[kOffW2 + j]);
      w2b[j] = b;
      w2tb[(j % kH) * kH + j / kH] = b;
    }
  }
}

// dst[c][m] = src[m][c] for m < n, zero for n <= m < ldT (BF16, 32 x 32 tiles)
__global__ void transpose_bf16_kernel(const uint16_t* __restrict__ src, unsigned long long n,
                                      int C, uint16_t* __restrict__ dst, unsigned long long ldT) {
  __shared__ uint16_t t[32][34];
  const unsigned long long m0 = (unsigned long long)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const unsigned long long m = m0 + r;
    t[r][threadIdx.x] = m < n ? src[m * C + c0 + threadIdx.x] : (uint16_t)0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const unsigned long long m = m0 + threadIdx.x;
    if (m < ldT) dst[(unsigned long long)(c0 + r) * ldT + m] = t[threadIdx.x][r];
  }
}

// counter-based He-normal init (splitmix64 + Box-Muller), zero biases
__device__ __forceinline__ unsigned long long splitmix(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__global__ void init_kernel(float* __restrict__ P, unsigned long long seed) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (int)kNumParams;
       i += gridDim.x * blockDim.x) {
    float fan_in;
    if (i < (int)kOffB1) fan_in = kIn;
    else if (i >= (int)kOffW2 && i < (int)kOffB2) fan_in = kH;
    else if (i >= (int)kOffW3 && i < (int)kOffB3) fan_in = kH;
    else {
      P[i] = 0.f;
      continue;
    }
    const unsigned long long h = splitmix(seed * 0x100000001B3ull + (unsigned long long)i);
    const float u1 = ((h >> 40) + 1) * (1.f / 16777217.f);
    const float u2 = ((h >> 16) & 0xFFFFFF) * (1.f / 16777216.f);
    const float z = sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
    P[i] = z * sqrtf(2.f / fan_in);
  }
}

// learned head: prediction -> position, residual test, plain fallback
// faces f in [f0, min(f0 + m, nn)); network rows at f - f0
__global__ void head_kernel(const __grid_constant__ FaceGeo geo, unsigned long long f0,
                            unsigned long long m, unsigned long long n,
                            const uint64_t* __restrict__ n_dev,
                            const uint64_t* __restrict__ face_ids,
                            const int8_t* __restrict__ winding, const float* __restrict__ yo,
                            const uint8_t* __restrict__ oko, const float* __restrict__ rmso,
                            float thresh, float* __restrict__ xyz, float* __restrict__ resid,
                            uint8_t* __restrict__ flags, unsigned long long* __restrict__ nfall) {
  unsigned long long nn = n;
  if (n_dev) nn = *n_dev < n ? *n_dev : n;
  if (f0 + m < nn) nn = f0 + m;
  unsigned int fallbacks = 0;
  for (unsigned long long f = f0 + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
       f < nn; f += (unsigned long long)gridDim.x * blockDim.x) {
    const GridGeo& G = geo.g[geo_snapshot(geo, f)];
    const float2* __restrict__ psi = G.psi;
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const float h = G.h, ox = G.ox, oy = G.oy, oz = G.oz;
    const unsigned long long row = f - f0;
    const uint64_t id = face_ids[f];
    const int wv = winding[f];
    bool use = oko[row] != 0 && (wv == 1 || wv == -1);
    const float u = yo[3 * row], v = yo[3 * row + 1];
    float r2 = 0.f;
    if (use) use = u >= -0.01f && u <= 1.01f && v >= -0.01f && v <= 1.01f;
    const int o = (int)(id & 3u);
    const unsigned long long lin = id >> 2;
    long long i, j, k;
    split_lin(lin, nx, ny, i, j, k);
    if (use) {
      const long long sx = 1, sy = nx, sz = (long long)nx * ny;
      const long long du = o == 0 ? sx : (o == 1 ? sy : sz);
      const long long dv = o == 0 ? sy : (o == 1 ? sz : sx);
      const float2 p0 = psi[lin], p1 = psi[lin + du], p2 = psi[lin + du + dv], p3 = psi[lin + dv];
      const float w0 = (1.f - u) * (1.f - v), w1 = u * (1.f - v), w2 = u * v, w3 = (1.f - u) * v;
      const float fr = w0 * p0.x + w1 * p1.x + w2 * p2.x + w3 * p3.x;
      const float fi = w0 * p0.y + w1 * p1.y + w2 * p2.y + w3 * p3.y;
      r2 = fr * fr + fi * fi;
      const float nr = rmso[row];
      use = r2 <= thresh * nr * nr;
    }
    if (use) {
      float gx = (float)i, gy = (float)j, gz = (float)k;
      if (o == 0) { gx += u; gy += v; }
      else if (o == 1) { gy += u; gz += v; }
      else { gz += u; gx += v; }
      xyz[3 * f] = fmaf(h, gx, ox);
      xyz[3 * f + 1] = fmaf(h, gy, oy);
      xyz[3 * f + 2] = fmaf(h, gz, oz);
      resid[f] = r2;
      flags[f] = QTV_FLAG_LEARNED;
    } else {
      float p[3], rr;
      uint8_t fl;
      loc::localize_face(psi, nx, ny, nz, h, ox, oy, oz, id, wv, p, &rr, &fl);
      xyz[3 * f] = p[0];
      xyz[3 * f + 1] = p[1];
      xyz[3 * f + 2] = p[2];
      resid[f] = rr;
      flags[f] = fl | QTV_FLAG_FALLBACK;
      ++fallbacks;
    }
  }
  for (int d = 16; d; d >>= 1) fallbacks += __shfl_xor_sync(0xffffffffu, fallbacks, d);
  if ((threadIdx.x & 31) == 0 && fallbacks && nfall) atomicAdd(nfall, (unsigned long long)fallbacks);
}

int blocks_for(unsigned long long n, int threads, int cap) {
  unsigned long long b = (n + threads - 1) / threads;
  if (b > (unsigned long long)cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

// ---------------------------------------------------------------------------
// Locator state owned by a handle
// ---------------------------------------------------------------------------
struct Locator {
  float* P = nullptr;      // parameters (FP32 master)
  float* G = nullptr;      // gradients
  float* M = nullptr;      // Adam first moment
  float* V = nullptr;      // Adam second moment
  uint16_t* w1b = nullptr; // BF16 W1 [256][128]
  uint16_t* w2b = nullptr; // BF16 W2 [256][256]
  uint16_t* w2tb = nullptr; // BF16 W2^T [256 in][256 out] (backward on tcgen05)
  unsigned long long step = 0;
  bool ready = false;
  // activations for up to `cap` rows; rows_gen counts their reallocations
  unsigned long long cap = 0;
  unsigned long long rows_gen = 0;
  // dense layers of forward passes: 0 = mma.sync kernel, 1 = tcgen05 kernel
  int tensor_path = 1;
  int num_sms = 0;
  unsigned int* status = nullptr;  // timeout flag of the tcgen05 kernel
  uint16_t *A1 = nullptr, *A2 = nullptr, *D1 = nullptr, *D2 = nullptr, *X = nullptr;
  // transposed copies for the weight gradients on tcgen05 ([features][ldT],
  // columns past the batch zero) and the split-K partials
  uint16_t *A1T = nullptr, *D1T = nullptr, *D2T = nullptr, *XT = nullptr;
  unsigned long long ldT = 0;
  float* part = nullptr;
  // per-block partials of the reductions over the batch: loss [1024], then
  // per 64-row chunk W3 and b3 (kOut kH + kOut), b2 and b1 (kH each)
  float* lpart = nullptr;
  float* gpart = nullptr;
  unsigned long long gpart_cap = 0;  // chunks
  float *Y = nullptr, *DY = nullptr, *rms = nullptr;
  uint8_t* ok = nullptr;
};

void locator_free(Locator* L) {
  if (!L) return;
  cudaFree(L->P);
  cudaFree(L->G);
  cudaFree(L->M);
  cudaFree(L->V);
  cudaFree(L->w1b);
  cudaFree(L->w2b);
  cudaFree(L->w2tb);
  cudaFree(L->A1T);
  cudaFree(L->D1T);
  cudaFree(L->D2T);
  cudaFree(L->XT);
  cudaFree(L->part);
  cudaFree(L->lpart);
  cudaFree(L->gpart);
  cudaFree(L->A1);
  cudaFree(L->A2);
  cudaFree(L->D1);
  cudaFree(L->D2);
  cudaFree(L->X);
  cudaFree(L->Y);
  cudaFree(L->DY);
  cudaFree(L->rms);
  cudaFree(L->ok);
  cudaFree(L->status);
  delete L;
}

static int locator_alloc(qtv_handle h) {
  if (h->loc) return QTV_OK;
  Locator* L = new (std::nothrow) Locator();
  if (!L) return set_error(QTV_ERR_ARG, "out of host memory");
  cudaError_t e = cudaSuccess;
  const size_t pb = kNumParams * sizeof(float);
  e = cudaMalloc(&L->P, pb);
  if (e == cudaSuccess) e = cudaMalloc(&L->G, pb);
  if (e == cudaSuccess) e = cudaMalloc(&L->M, pb);
  if (e == cudaSuccess) e = cudaMalloc(&L->V, pb);
  if (e == cudaSuccess) e = cudaMalloc(&L->w1b, (size_t)kH * kIn * 2);
  if (e == cudaSuccess) e = cudaMalloc(&L->w2b, (size_t)kH * kH * 2);
  if (e == cudaSuccess) e = cudaMalloc(&L->w2tb, (size_t)kH * kH * 2);
  if (e == cudaSuccess) e = cudaMalloc(&L->part, (size_t)kSplits * kH * kH * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&L->lpart, (size_t)kLossBlocks * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&L->status, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(L->status, 0, sizeof(unsigned int));
  if (e != cudaSuccess) {
    locator_free(L);
    return check_cuda(e, "cudaMalloc(locator)");
  }
  L->num_sms = h->num_sms;
  h->loc = L;
  return QTV_OK;
}

static int locator_rows(qtv_handle h, unsigned long long n, cudaStream_t st) {
  Locator* L = h->loc;
  if (n <= L->cap) return QTV_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
    return set_error(QTV_ERR_STATE, "locator buffers must grow during stream capture");
  cudaFree(L->A1);
  cudaFree(L->A2);
  cudaFree(L->D1);
  cudaFree(L->D2);
  cudaFree(L->X);
  cudaFree(L->Y);
  cudaFree(L->DY);
  cudaFree(L->rms);
  cudaFree(L->ok);
  cudaFree(L->A1T);
  cudaFree(L->D1T);
  cudaFree(L->D2T);
  cudaFree(L->XT);
  L->A1T = L->D1T = L->D2T = L->XT = nullptr;
  L->A1 = L->A2 = L->D1 = L->D2 = L->X = nullptr;
  L->Y = L->DY = L->rms = nullptr;
  L->ok = nullptr;
  L->cap = 0;
  cudaError_t e = cudaMalloc(&L->A1, n * kH * 2);
  if (e == cudaSuccess) e = cudaMalloc(&L->A2, n * kH * 2);
  if (e == cudaSuccess) e = cudaMalloc(&L->D1, n * kH * 2);
  if (e == cudaSuccess) e = cudaMalloc(&L->D2, n * kH * 2);
  if (e == cudaSuccess) e = cudaMalloc(&L->X, n * kIn * 2);
  if (e == cudaSuccess) e = cudaMalloc(&L->Y, n * kOut * 4);
  if (e == cudaSuccess) e = cudaMalloc(&L->DY, n * kOut * 4);
  if (e == cudaSuccess) e = cudaMalloc(&L->rms, n * 4);
  if (e == cudaSuccess) e = cudaMalloc(&L->ok, n);
  const unsigned long long ldT = (n + 63) / 64 * 64;
  if (e == cudaSuccess) e = cudaMalloc(&L->A1T, ldT * kH * 2);
  if (e == cudaSuccess) e = cudaMalloc(&L->D1T, ldT * kH * 2);
  if (e == cudaSuccess) e = cudaMalloc(&L->D2T, ldT * kH * 2);
  if (e == cudaSuccess) e = cudaMalloc(&L->XT, ldT * kIn * 2);
  if (e != cudaSuccess) return check_cuda(e, "cudaMalloc(locator rows)");
  L->ldT = ldT;
  L->cap = n;
  ++L->rows_gen;
  return QTV_OK;
}

static int forward_hidden(Locator* L, const uint16_t* X, unsigned long long n, cudaStream_t st) {
  int rc = gemm<false, false, EPI_BIAS_RELU_BF16>((int)n, kH, kIn, X, kIn, L->w1b, kIn, L->A1, kH,
                                                  L->P + kOffB1, nullptr, st);
  if (rc) return rc;
  return gemm<false, false, EPI_BIAS_RELU_BF16>((int)n, kH, kH, L->A1, kH, L->w2b, kH, L->A2, kH,
                                                L->P + kOffB2, nullptr, st);
}

// network outputs Y[n][3] of inputs X (forward passes of inference)
static int forward_y(Locator* L, const uint16_t* X, unsigned long long n, float* Y,
                     cudaStream_t st) {
  if (L->tensor_path == 1)
    return tc_mlp_forward(X, (long long)n, L->w1b, L->w2b, L->P + kOffB1, L->P + kOffB2,
                          L->P + kOffW3, L->P + kOffB3, Y, L->status, L->num_sms, st);
  int rc = forward_hidden(L, X, n, st);
  if (rc) return rc;
  out_layer_kernel<<<blocks_for(n, 256, 4096), 256, 0, st>>>(L->A2, L->P, n, Y, nullptr, nullptr,
                                                              nullptr);
  return check_cuda(cudaGetLastError(), "out_layer_kernel launch");
}

// the partial buffers of the batch reductions for n rows
static int grad_parts(Locator* L, unsigned long long n, cudaStream_t st) {
  const unsigned long long chunks = (n + kRowChunk - 1) / kRowChunk;
  if (chunks <= L->gpart_cap) return QTV_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
    return set_error(QTV_ERR_STATE, "locator buffers must grow during stream capture");
  cudaFree(L->gpart);
  L->gpart = nullptr;
  L->gpart_cap = 0;
  const cudaError_t e = cudaMalloc(&L->gpart, chunks * (kPartW3 + 2 * kH) * sizeof(float));
  if (e != cudaSuccess) return check_cuda(e, "cudaMalloc(gradient partials)");
  L->gpart_cap = chunks;
  return QTV_OK;
}

// output layer with loss and dY, its weight gradients, and the loss summed in
// block order (the first half of the backward pass, both tensor paths)
static int output_backward(Locator* L, const float* T, unsigned long long n, float* loss,
                           cudaStream_t st) {
  const int nbl = blocks_for(n, 256, kLossBlocks);
  out_layer_kernel<<<nbl, 256, 0, st>>>(L->A2, L->P, n, L->Y, T, L->DY, L->lpart);
  sum_parts_kernel<<<1, 32, 0, st>>>(L->lpart, nbl, 1, loss);
  out_back_kernel<<<blocks_for(n * kH, 256, 4096), 256, 0, st>>>(L->DY, L->P, L->A2, n, L->D2);
  const unsigned chunks = (unsigned)((n + kRowChunk - 1) / kRowChunk);
  float* p3 = L->gpart;
  out_wgrad_kernel<<<chunks, kH + 32, 0, st>>>(L->DY, L->A2, n, p3);
  sum_parts_kernel<<<4, 256, 0, st>>>(p3, (int)chunks, kPartW3, L->G + kOffW3);
  return check_cuda(cudaGetLastError(), "locator output backward");
}

// bias gradient of a layer: column sums of dH (BF16 [n][kH]) in block order
static int bias_grad(Locator* L, const uint16_t* D, unsigned long long n, int which, float* out,
                     cudaStream_t st) {
  const unsigned chunks = (unsigned)((n + kRowChunk - 1) / kRowChunk);
  float* p = L->gpart + (size_t)L->gpart_cap * kPartW3 + (size_t)which * L->gpart_cap * kH;
  colsum_kernel<<<chunks, kH, 0, st>>>(D, n, p);
  sum_parts_kernel<<<1, kH, 0, st>>>(p, (int)chunks, kH, out);
  return check_cuda(cudaGetLastError(), "locator bias gradient");
}

// splits of a K range of k64 chunks of 64: the largest divisor up to kSplits
static int splits_for(unsigned long long k64) {
  int s = kSplits;
  while (s > 1 && k64 % (unsigned long long)s) --s;
  return s;
}

// forward + backward into L->G on tcgen05 (L->tensor_path == 1): the dense
// layers and the data-gradient GEMM take the row-major activations, the
// weight-gradient GEMMs the transposed copies (K = the padded batch, split
// into parts summed in a fixed order)
static int forward_backward_tc(Locator* L, const uint16_t* X, const float* T, unsigned long long n,
                               float* loss, cudaStream_t st) {
  const unsigned long long ldT = (n + 63) / 64 * 64;
  const dim3 tb(32, 8);
  transpose_bf16_kernel<<<dim3((unsigned)(ldT / 32), kIn / 32), tb, 0, st>>>(X, n, kIn, L->XT, ldT);
  // A1 = relu(X W1^T + b1), and A1^T
  cudaError_t e = cudaSuccess;
  if (ldT > n) {  // the GEMM epilogues write columns below n only
    e = cudaMemset2DAsync(L->A1T + n, ldT * 2, 0, (ldT - n) * 2, kH, st);
    if (e == cudaSuccess) e = cudaMemset2DAsync(L->D1T + n, ldT * 2, 0, (ldT - n) * 2, kH, st);
    if (e != cudaSuccess) return check_cuda(e, "memset(transposed padding)");
  }
  int rc = tc_gemm(X, kIn, L->w1b, kIn, (long long)n, kH, kIn, 1, 1, nullptr, 0, nullptr, L->A1, kH,
                   L->A1T, (long long)ldT, L->P + kOffB1, nullptr, 0, L->status, st);
  if (rc) return rc;
  // A2 = relu(A1 W2^T + b2)
  rc = tc_gemm(L->A1, kH, L->w2b, kH, (long long)n, kH, kH, 1, 1, nullptr, 0, nullptr, L->A2, kH,
               nullptr, 0, L->P + kOffB2, nullptr, 0, L->status, st);
  if (rc) return rc;
  rc = output_backward(L, T, n, loss, st);
  if (rc) return rc;
  transpose_bf16_kernel<<<dim3((unsigned)(ldT / 32), kH / 32), tb, 0, st>>>(L->D2, n, kH, L->D2T, ldT);
  rc = bias_grad(L, L->D2, n, 0, L->G + kOffB2, st);
  if (rc) return rc;
  const int sp = splits_for(ldT / 64);
  // dW2[o][k] = sum_m dH2[m][o] A1[m][k]
  rc = tc_gemm(L->D2T, (long long)ldT, L->A1T, (long long)ldT, kH, kH, (long long)ldT, sp, 0,
               L->G + kOffW2, kH, L->part, nullptr, 0, nullptr, 0, nullptr, nullptr, 0, L->status, st);
  if (rc) return rc;
  // dH1[m][k] = (sum_o dH2[m][o] W2[o][k]) * (A1[m][k] > 0), and its transpose
  rc = tc_gemm(L->D2, kH, L->w2tb, kH, (long long)n, kH, kH, 1, 2, nullptr, 0, nullptr, L->D1, kH,
               L->D1T, (long long)ldT, nullptr, L->A1, kH, L->status, st);
  if (rc) return rc;
  rc = bias_grad(L, L->D1, n, 1, L->G + kOffB1, st);
  if (rc) return rc;
  // dW1[o][i] = sum_m dH1[m][o] X[m][i]
  rc = tc_gemm(L->D1T, (long long)ldT, L->XT, (long long)ldT, kH, kIn, (long long)ldT, sp, 0,
               L->G + kOffW1, kIn, L->part, nullptr, 0, nullptr, 0, nullptr, nullptr, 0, L->status,
               st);
  if (rc) return rc;
  return check_cuda(cudaGetLastError(), "locator backward (tcgen05)");
}

// forward + backward into L->G; loss (device float) accumulated
static int forward_backward(Locator* L, const uint16_t* X, const float* T, unsigned long long n,
                            float* loss, cudaStream_t st) {
  int rc = grad_parts(L, n, st);
  if (rc) return rc;
  if (L->tensor_path == 1) return forward_backward_tc(L, X, T, n, loss, st);
  rc = forward_hidden(L, X, n, st);
  if (rc) return rc;
  rc = output_backward(L, T, n, loss, st);
  if (rc) return rc;
  rc = bias_grad(L, L->D2, n, 0, L->G + kOffB2, st);
  if (rc) return rc;
  // dW2[n][k] = sum_m dH2[m][n] A1[m][k]
  rc = gemm<true, true, EPI_STORE_F32>(kH, kH, (int)n, L->D2, kH, L->A1, kH, L->G + kOffW2, kH,
                                       nullptr, nullptr, st);
  if (rc) return rc;
  // dH1[m][k] = (sum_n dH2[m][n] W2[n][k]) * (A1 > 0)
  rc = gemm<false, true, EPI_RELU_MASK_BF16>((int)n, kH, kH, L->D2, kH, L->w2b, kH, L->D1, kH,
                                             nullptr, L->A1, st);
  if (rc) return rc;
  rc = bias_grad(L, L->D1, n, 1, L->G + kOffB1, st);
  if (rc) return rc;
  // dW1[n][k] = sum_m dH1[m][n] X[m][k]
  rc = gemm<true, true, EPI_STORE_F32>(kH, kIn, (int)n, L->D1, kH, X, kIn, L->G + kOffW1, kIn,
                                       nullptr, nullptr, st);
  if (rc) return rc;
  return check_cuda(cudaGetLastError(), "locator backward");
}

constexpr unsigned long long kLocChunk = 1ull << 20;  // faces per learned chunk

int locator_prepare(qtv_handle h, uint64_t n, uint64_t* generation) {
  Locator* L = h->loc;
  if (!L || !L->ready) return set_error(QTV_ERR_STATE, "no learned locator loaded");
  const int rc = locator_rows(h, n < kLocChunk ? n : kLocChunk, nullptr);
  if (generation) *generation = L->rows_gen;
  return rc;
}

int locator_localize(qtv_handle h, const FaceGeo& geo, const uint64_t* face_ids,
                     const int8_t* winding, uint64_t n, const uint64_t* n_dev, float thresh,
                     float* xyz, float* resid, uint8_t* flags, cudaStream_t st) {
  Locator* L = h->loc;
  if (!L || !L->ready) return set_error(QTV_ERR_STATE, "no learned locator loaded");
  const unsigned long long chunk = n < kLocChunk ? n : kLocChunk;
  int rc = locator_rows(h, chunk, st);
  if (rc) return rc;
  for (unsigned long long f0 = 0; f0 < n; f0 += chunk) {
    const unsigned long long m = n - f0 < chunk ? n - f0 : chunk;
    {
      TraceScope ts(h, K_ENCODE, st);
      encode_kernel<<<blocks_for((m + kEncFacesPerWarp - 1) / kEncFacesPerWarp * 32, 256, 65535), 256, 0,
                      st>>>(
          geo, f0, m, n, n_dev, face_ids, winding, L->X, L->ok, L->rms);
    }
    {
      TraceScope ts(h, K_NETWORK, st);
      rc = forward_y(L, L->X, m, L->Y, st);
    }
    if (rc) return rc;
    TraceScope ts(h, K_HEAD, st);
    head_kernel<<<blocks_for(m, 256, 65535), 256, 0, st>>>(geo, f0, m, n, n_dev, face_ids, winding,
                                                           L->Y, L->ok, L->rms, thresh, xyz, resid,
                                                           flags, nullptr);
  }
  return check_cuda(cudaGetLastError(), "learned localize");
}

}  // namespace qtv

using namespace qtv;

extern "C" {

int qtv_locator_init(qtv_handle h, uint64_t seed) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  int rc = locator_alloc(h);
  if (rc) return rc;
  Locator* L = h->loc;
  init_kernel<<<64, 256>>>(L->P, seed);
  cudaMemset(L->M, 0, kNumParams * 4);
  cudaMemset(L->V, 0, kNumParams * 4);
  refresh_bf16_kernel<<<64, 256>>>(L->P, L->w1b, L->w2b, L->w2tb);
  L->step = 0;
  L->ready = true;
  return check_cuda(cudaDeviceSynchronize(), "qtv_locator_init");
}

int qtv_locator_set_tensor_path(qtv_handle h, int path) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  if (path != 0 && path != 1) return set_error(QTV_ERR_ARG, "tensor path %d (0 or 1)", path);
  int rc = locator_alloc(h);
  if (rc) return rc;
  h->loc->tensor_path = path;
  return QTV_OK;
}

int qtv_locator_get(qtv_handle h, float* params, float* adam, uint64_t* step) {
  if (!h || !h->loc || !h->loc->ready) return set_error(QTV_ERR_STATE, "no learned locator loaded");
  Locator* L = h->loc;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && params) e = cudaMemcpy(params, L->P, kNumParams * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && adam) e = cudaMemcpy(adam, L->M, kNumParams * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && adam)
    e = cudaMemcpy(adam + kNumParams, L->V, kNumParams * 4, cudaMemcpyDeviceToHost);
  if (step) *step = L->step;
  return check_cuda(e, "qtv_locator_get");
}

int qtv_locator_set(qtv_handle h, const float* params, const float* adam, uint64_t step) {
  if (!h || !params) return set_error(QTV_ERR_ARG, "handle or params is NULL");
  int rc = locator_alloc(h);
  if (rc) return rc;
  Locator* L = h->loc;
  cudaError_t e = cudaMemcpy(L->P, params, kNumParams * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    if (adam) {
      e = cudaMemcpy(L->M, adam, kNumParams * 4, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(L->V, adam + kNumParams, kNumParams * 4, cudaMemcpyHostToDevice);
    } else {
      e = cudaMemset(L->M, 0, kNumParams * 4);
      if (e == cudaSuccess) e = cudaMemset(L->V, 0, kNumParams * 4);
    }
  }
  if (e != cudaSuccess) return check_cuda(e, "qtv_locator_set");
  refresh_bf16_kernel<<<64, 256>>>(L->P, L->w1b, L->w2b, L->w2tb);
  L->step = step;
  L->ready = true;
  return check_cuda(cudaDeviceSynchronize(), "qtv_locator_set");
}

int qtv_locator_encode(qtv_handle h, const qtv_grid* grid, const void* psi, const uint64_t* face_ids,
                       const int8_t* winding, uint64_t n, const uint64_t* n_dev, uint16_t* x,
                       uint8_t* ok, float* rms, void* stream) {
  if (!h || !grid) return set_error(QTV_ERR_ARG, "handle or grid is NULL");
  if (n == 0) return QTV_OK;
  if (!psi || !face_ids || !winding || !x || !ok || !rms)
    return set_error(QTV_ERR_ARG, "a required pointer is NULL");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  encode_kernel<<<blocks_for((n + kEncFacesPerWarp - 1) / kEncFacesPerWarp * 32, 256, 65535), 256,
                  0, st>>>(
      single_geo(*grid, reinterpret_cast<const float2*>(psi)), 0ull, n, n, n_dev, face_ids,
      winding, x, ok, rms);
  return check_cuda(cudaGetLastError(), "encode_kernel launch");
}

int qtv_locator_forward(qtv_handle h, const uint16_t* x, uint64_t n, float* y, void* stream) {
  if (!h || !h->loc || !h->loc->ready) return set_error(QTV_ERR_STATE, "no learned locator loaded");
  if (n == 0) return QTV_OK;
  if (!x || !y) return set_error(QTV_ERR_ARG, "x or y is NULL");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int rc = locator_rows(h, n, st);
  if (rc) return rc;
  return forward_y(h->loc, x, n, y, st);
}

int qtv_locator_gradients(qtv_handle h, const uint16_t* x, const float* targets, uint64_t n,
                          float* grads, float* loss, void* stream) {
  if (!h || !h->loc || !h->loc->ready) return set_error(QTV_ERR_STATE, "no learned locator loaded");
  if (!x || !targets || !loss || n == 0 || n % 64)
    return set_error(QTV_ERR_ARG, "x/targets/loss NULL or batch not a positive multiple of 64");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int rc = locator_rows(h, n, st);
  if (rc) return rc;
  cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), st);
  if (e != cudaSuccess) return check_cuda(e, "memset(loss)");
  rc = forward_backward(h->loc, x, targets, n, loss, st);
  if (rc) return rc;
  if (grads)
    return check_cuda(cudaMemcpyAsync(grads, h->loc->G, kNumParams * 4, cudaMemcpyDeviceToDevice, st),
                      "copy(grads)");
  return QTV_OK;
}

int qtv_locator_train_step(qtv_handle h, const uint16_t* x, const float* targets, uint64_t n,
                           float lr, float* loss, void* stream) {
  int rc = qtv_locator_gradients(h, x, targets, n, nullptr, loss, stream);
  if (rc) return rc;
  Locator* L = h->loc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  L->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)L->step), c2 = 1.f - powf(b2, (float)L->step);
  adam_kernel<<<128, 256, 0, st>>>(L->P, L->G, L->M, L->V, (int)kNumParams, lr, b1, b2, 1e-8f, c1,
                                   c2, L->w1b, L->w2b, L->w2tb);
  return check_cuda(cudaGetLastError(), "adam_kernel launch");
}

// Checkpoint: magic, version, step, parameters, Adam moments, FNV-1a checksum.
int qtv_locator_save(qtv_handle h, const char* path) {
  if (!path) return set_error(QTV_ERR_ARG, "path is NULL");
  std::vector<float> buf(3 * kNumParams);
  uint64_t step = 0;
  int rc = qtv_locator_get(h, buf.data(), buf.data() + kNumParams, &step);
  if (rc) return rc;
  uint64_t hsh = 1469598103934665603ull;
  const unsigned char* bytes = reinterpret_cast<const unsigned char*>(buf.data());
  for (size_t i = 0; i < buf.size() * 4; ++i) hsh = (hsh ^ bytes[i]) * 1099511628211ull;
  FILE* fp = fopen(path, "wb");
  if (!fp) return set_error(QTV_ERR_ARG, "cannot open %s for writing", path);
  const uint32_t head[2] = {0x31565451u, 1u};  // "QTV1", version 1
  const uint64_t np = kNumParams;
  bool ok = fwrite(head, sizeof head, 1, fp) == 1 && fwrite(&np, 8, 1, fp) == 1 &&
            fwrite(&step, 8, 1, fp) == 1 && fwrite(buf.data(), 4, buf.size(), fp) == buf.size() &&
            fwrite(&hsh, 8, 1, fp) == 1;
  ok = fclose(fp) == 0 && ok;
  return ok ? QTV_OK : set_error(QTV_ERR_ARG, "short write to %s", path);
}

int qtv_locator_load(qtv_handle h, const char* path) {
  if (!path) return set_error(QTV_ERR_ARG, "path is NULL");
  FILE* fp = fopen(path, "rb");
  if (!fp) return set_error(QTV_ERR_ARG, "cannot open %s", path);
  uint32_t head[2];
  uint64_t np = 0, step = 0, hsh = 0;
  std::vector<float> buf(3 * kNumParams);
  bool ok = fread(head, sizeof head, 1, fp) == 1 && fread(&np, 8, 1, fp) == 1 &&
            fread(&step, 8, 1, fp) == 1;
  ok = ok && head[0] == 0x31565451u && head[1] == 1u && np == kNumParams;
  ok = ok && fread(buf.data(), 4, buf.size(), fp) == buf.size() && fread(&hsh, 8, 1, fp) == 1;
  fclose(fp);
  if (!ok) return set_error(QTV_ERR_ARG, "%s is not a locator checkpoint", path);
  uint64_t chk = 1469598103934665603ull;
  const unsigned char* bytes = reinterpret_cast<const unsigned char*>(buf.data());
  for (size_t i = 0; i < buf.size() * 4; ++i) chk = (chk ^ bytes[i]) * 1099511628211ull;
  if (chk != hsh) return set_error(QTV_ERR_ARG, "%s: checksum mismatch", path);
  return qtv_locator_set(h, buf.data(), buf.data() + kNumParams, step);
}

}  // extern "C"
