// locator_tc.cu -- the learned locator's network on the 5th-generation tensor
// cores (tcgen05, accumulators in tensor memory): a dense layer
// out[M][256] = relu(A[M][K] W[256][K]^T + b) in BF16 (K = 128 or 256), and
// the whole 128-256-256-3 network fused per 128-row tile (tc_mlp_kernel).
//
// A persistent CTA of 4 warps keeps W in shared memory for all its 128-row
// tiles of A.  Operands are stored in the canonical K-major layout without
// swizzle: 8 x 8 core matrices of 128 contiguous bytes (8 rows of 16 bytes),
// core matrix (r / 8, k / 8) at ((r / 8) (K / 8) + k / 8) 128 bytes, so the
// leading-dimension offset (next core matrix along K) is 128 bytes and the
// stride offset (next 8-row group) is 16 K bytes.  One elected thread issues
// K / 16 tcgen05.mma instructions of M = 128, N = 256, K = 16 into a 256-column
// FP32 accumulator in tensor memory and commits them to an mbarrier; then each
// warp reads its 32 rows back with tcgen05.ld (32 columns at a time), adds the
// bias, applies ReLU, rounds to BF16 and stores 64 contiguous bytes per row.
// The accumulator columns are allocated once per CTA and freed before exit;
// the mbarrier wait is bounded and sets a status flag on timeout.
#include <cuda_bf16.h>

#include "qtv_internal.cuh"
#include "sweep_common.cuh"

namespace qtv {
namespace {

using namespace sweep;

constexpr int TM = 128;   // rows per tile (M of one instruction, TMEM lanes)
constexpr int TN = 256;   // outputs (N of one instruction, TMEM columns)

__device__ __forceinline__ uint32_t bf16x2_bits(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// shared-memory matrix descriptor: no swizzle, K-major
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the 5th-generation tensor cores
  return d;                // base offset 0, swizzle none
}

// instruction descriptor of kind::f16: D F32, A and B BF16, both K-major
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

// rows [r0, r0 + R) of a row-major BF16 matrix (K columns, row pitch K) into
// the canonical layout at dst; rows at or beyond nrows become zero.  Piece c
// (16 bytes) goes to byte 16 c of dst: c = ((r / 8) (K / 8) + k / 8) 8 + r % 8,
// so consecutive threads fill consecutive shared-memory slots (no bank
// conflicts) and read 8 rows x 16 bytes per group of 8 threads.
__device__ __forceinline__ void load_canon(unsigned char* dst, const uint16_t* __restrict__ src,
                                           long long r0, int R, long long nrows, int K) {
  const int kc8 = K / 8;
  const int chunks = R * kc8;
  for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
    const int rr = c & 7, kc = (c >> 3) % kc8, rg = (c >> 3) / kc8;
    const int r = rg * 8 + rr;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (r0 + r < nrows) v = __ldg(reinterpret_cast<const uint4*>(src + (r0 + r) * K) + kc);
    *reinterpret_cast<uint4*>(dst + (size_t)c * 16) = v;
  }
}

// as load_canon, with cp.async (16 bytes per piece, zero fill past nrows);
// completion by cp_async_wait_all
__device__ __forceinline__ void load_canon_async(unsigned char* dst, const uint16_t* __restrict__ src,
                                                 long long r0, int R, long long nrows, int K) {
  const int kc8 = K / 8;
  const int chunks = R * kc8;
  for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
    const int rr = c & 7, kc = (c >> 3) % kc8, rg = (c >> 3) / kc8;
    const long long r = r0 + rg * 8 + rr;
    const bool in = r < nrows;
    const uint16_t* g = src + (in ? r : 0) * K + kc * 8;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst + (size_t)c * 16)),
                 "l"(g), "r"(in ? 16 : 0)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

__global__ void __launch_bounds__(128, 1) tc_dense_kernel(const uint16_t* __restrict__ A,
                                                          long long M, int K,
                                                          const uint16_t* __restrict__ W,
                                                          const float* __restrict__ bias,
                                                          uint16_t* __restrict__ out,
                                                          unsigned int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  unsigned char* sW = dsm;                                 // TN x K
  unsigned char* sA = dsm + (size_t)TN * K * 2;            // TM x K
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sA + (size_t)TM * K * 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  float* sb = reinterpret_cast<float*>(tslot + 4);         // bias [TN]
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;

  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"((uint32_t)TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(mbar, 1u);
    fence_mbar_init();
  }
  for (int i = tid; i < TN; i += blockDim.x) sb[i] = bias[i];
  load_canon(sW, W, 0, TN, TN, K);
  fence_proxy_async();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t lbo = 128u, sbo = (uint32_t)(K / 8) * 128u;
  const uint64_t adesc0 = smem_desc(smem_u32(sA), lbo, sbo);
  const uint64_t bdesc0 = smem_desc(smem_u32(sW), lbo, sbo);
  bool timeout = false;
  uint32_t phase = 0;

  const long long ntiles = (M + TM - 1) / TM;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long r0 = tile * TM;
    load_canon(sA, A, r0, TM, M, K);
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int kb = 0; kb < K / 16; ++kb) {
        // advance both start addresses by two core matrices (256 bytes) per K step
        const uint64_t adv = (uint64_t)((kb * 256) >> 4);
        const uint32_t acc = kb > 0 ? 1u : 0u;
        asm volatile(
            "{\n"
            " .reg .pred p;\n"
            " setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
            "}\n" ::"r"(tmem),
            "l"(adesc0 + adv), "l"(bdesc0 + adv), "r"(kIdesc), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(mbar))
          : "memory");
    }
    if (!mbar_wait(mbar, phase)) timeout = true;
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: warp w owns TMEM lanes (rows) 32 w .. 32 w + 31
    const long long row = r0 + 32 * w + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < TN; c0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(32 * w) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
          "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
          "%28, %29, %30, %31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
            "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
            "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < M) {
        uint32_t pk[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float lo = fmaxf(__uint_as_float(v[2 * j]) + sb[c0 + 2 * j], 0.f);
          const float hi = fmaxf(__uint_as_float(v[2 * j + 1]) + sb[c0 + 2 * j + 1], 0.f);
          pk[j] = bf16x2_bits(lo, hi);
        }
        uint4* dst = reinterpret_cast<uint4*>(out + row * TN + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          dst[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (timeout) atomicOr(status, 1u);
  __syncthreads();
  if (w == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)TN)
                 : "memory");
}

// ---------------------------------------------------------------------------
// The whole network for 128-row tiles: Y[M][3] = W3 relu(W2 relu(W1 x + b1) +
// b2) + b3.  W1 (64 KB) and W2 (128 KB) stay in shared memory; per tile the X
// rows (32 KB) are loaded, layer 1 accumulates into TMEM columns [0, 256),
// its epilogue writes relu(. + b1) as BF16 pairs back into TMEM columns
// [0, 128) (row = lane, two consecutive K values per 32-bit column), layer 2
// takes that A operand from TMEM and accumulates into columns [256, 512), and
// its epilogue applies relu(. + b2) and the 3-output layer in FP32.  The next
// tile's X is prefetched with cp.async once layer 1 has read the current one,
// and the next tile's layer 1 runs on the tensor cores during epilogue 2.
// Eight warps: warps w and w + 4 read the same 32 TMEM lanes (rows) and split
// the columns, so each SM sub-partition has two warps to hide tcgen05.ld
// latency; the upper half's partial 3-output sums meet the lower half's in
// shared memory.
// ---------------------------------------------------------------------------
constexpr uint32_t kMlpSmemW1 = 256 * 128 * 2, kMlpSmemW2 = 256 * 256 * 2, kMlpSmemX = 128 * 128 * 2;
constexpr int kMlpThreads = 256;
constexpr uint32_t kMlpSmemPart = TM * 3 * sizeof(float);  // upper-half partial outputs

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
      "r"(v[15])
      : "memory");
}

__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__global__ void __launch_bounds__(kMlpThreads, 1) tc_mlp_kernel(
    const uint16_t* __restrict__ X, long long M, const uint16_t* __restrict__ W1,
    const uint16_t* __restrict__ W2, const float* __restrict__ b1, const float* __restrict__ b2,
    const float* __restrict__ w3, const float* __restrict__ b3, float* __restrict__ Y,
    unsigned int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  unsigned char* sW1 = dsm;
  unsigned char* sW2 = dsm + kMlpSmemW1;
  unsigned char* sX = sW2 + kMlpSmemW2;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sX + kMlpSmemX);  // layer 1 done
  uint64_t* mbar2 = mbar + 1;                                          // layer 2 done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  float* spart = reinterpret_cast<float*>(sX + kMlpSmemX + 32);  // [TM][3]
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int wq = w & 3;      // TMEM lane quarter (rows 32 wq .. 32 wq + 31)
  const int half = w >> 2;   // column half of the epilogues

  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(mbar, 1u);
    mbar_init(mbar2, 1u);
    fence_mbar_init();
  }
  load_canon(sW1, W1, 0, 256, 256, 128);
  load_canon(sW2, W2, 0, 256, 256, 256);
  fence_proxy_async();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t lane_off = (uint32_t)(32 * wq) << 16;
  const uint64_t xdesc = smem_desc(smem_u32(sX), 128u, 16u * 128u);
  const uint64_t w1desc = smem_desc(smem_u32(sW1), 128u, 16u * 128u);
  const uint64_t w2desc = smem_desc(smem_u32(sW2), 128u, 32u * 128u);
  bool timeout = false;
  uint32_t phase = 0;

  const long long ntiles = (M + TM - 1) / TM;
  uint32_t phase2 = 0;
  auto issue_layer1 = [&]() {  // D1 (columns 0..255) = X W1^T, 8 steps of K = 16
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int kb = 0; kb < 8; ++kb)
        mma_ss(tmem, xdesc + (uint64_t)(kb * 16), w1desc + (uint64_t)(kb * 16), kb > 0 ? 1u : 0u);
      mma_commit(mbar);
    }
  };
  if ((long long)blockIdx.x < ntiles) {
    load_canon_async(sX, X, (long long)blockIdx.x * TM, TM, M, 128);
    cp_async_wait_all();
    fence_proxy_async();
    __syncthreads();
    issue_layer1();
  }
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long r0 = tile * TM;
    const long long row = r0 + 32 * wq + lane;
    const long long next = tile + gridDim.x;
    if (!mbar_wait(mbar, phase)) timeout = true;  // layer 1 of this tile
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // X of the next tile streams into shared memory during the rest of this tile
    if (next < ntiles) load_canon_async(sX, X, next * TM, TM, M, 128);
    // epilogue 1: columns 32 j .. 32 j + 31 of D1 -> BF16 pairs in columns 16 j .. 16 j + 15,
    // this warp's half j = 4 half .. 4 half + 3.  The pairs of block j land on D1 columns that
    // block j / 2 reads, which may be the other half's, so every warp reads all its blocks
    // before any warp writes.
    // (the bias of column 32 j + i is lane i's coalesced load, broadcast by a
    // shuffle: one load per block instead of eight per lane)
    uint32_t pk[4][16];
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int j = 4 * half + jj;
      const float lb = __ldg(b1 + 32 * j + lane);
      uint32_t v[32];
      tmem_ld32(tmem + lane_off + 32u * j, v);
#pragma unroll
      for (int i = 0; i < 32; i += 2)
        pk[jj][i / 2] =
            bf16x2_bits(fmaxf(__uint_as_float(v[i]) + __shfl_sync(0xffffffffu, lb, i), 0.f),
                        fmaxf(__uint_as_float(v[i + 1]) + __shfl_sync(0xffffffffu, lb, i + 1), 0.f));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) tmem_st16(tmem + lane_off + 16u * (4 * half + jj), pk[jj]);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // layer 2: D2 (columns 256..511) = A1 W2^T, A1 from TMEM columns 8 kb .. 8 kb + 7
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int kb = 0; kb < 16; ++kb)
        mma_ts(tmem + 256u, tmem + 8u * kb, w2desc + (uint64_t)(kb * 16), kb > 0 ? 1u : 0u);
      mma_commit(mbar2);
    }
    if (!mbar_wait(mbar2, phase2)) timeout = true;
    phase2 ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // layer 1 of the next tile runs on the tensor cores during epilogue 2
    // (D1 and A1 are free now; its X is complete and visible)
    cp_async_wait_all();
    fence_proxy_async();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (next < ntiles) issue_layer1();
    // epilogue 2: relu(. + b2) and the 3-output layer in FP32
    float y0 = 0.f, y1 = 0.f, y2 = 0.f;
#pragma unroll 1
    for (int j = 4 * half; j < 4 * half + 4; ++j) {
      // bias and output weights of column 32 j + i: lane i's loads, broadcast
      const float lb = __ldg(b2 + 32 * j + lane), l0 = __ldg(w3 + 32 * j + lane),
                  l1 = __ldg(w3 + 256 + 32 * j + lane), l2 = __ldg(w3 + 512 + 32 * j + lane);
      uint32_t v[32];
      tmem_ld32(tmem + lane_off + 256u + 32u * j, v);
#pragma unroll
      for (int i4 = 0; i4 < 8; ++i4) {
        float a[4], c0[4], c1[4], c2[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int i = 4 * i4 + e;
          a[e] = fmaxf(__uint_as_float(v[i]) + __shfl_sync(0xffffffffu, lb, i), 0.f);
          c0[e] = __shfl_sync(0xffffffffu, l0, i);
          c1[e] = __shfl_sync(0xffffffffu, l1, i);
          c2[e] = __shfl_sync(0xffffffffu, l2, i);
        }
        y0 = fmaf(c0[0], a[0], fmaf(c0[1], a[1], fmaf(c0[2], a[2], fmaf(c0[3], a[3], y0))));
        y1 = fmaf(c1[0], a[0], fmaf(c1[1], a[1], fmaf(c1[2], a[2], fmaf(c1[3], a[3], y1))));
        y2 = fmaf(c2[0], a[0], fmaf(c2[1], a[1], fmaf(c2[2], a[2], fmaf(c2[3], a[3], y2))));
      }
    }
    // the upper column half's partial sums join the lower half's
    const int rl = 32 * wq + lane;
    if (half) {
      spart[3 * rl] = y0;
      spart[3 * rl + 1] = y1;
      spart[3 * rl + 2] = y2;
    }
    __syncthreads();
    if (!half && row < M) {
      Y[3 * row] = (y0 + spart[3 * rl]) + __ldg(b3);
      Y[3 * row + 1] = (y1 + spart[3 * rl + 1]) + __ldg(b3 + 1);
      Y[3 * row + 2] = (y2 + spart[3 * rl + 2]) + __ldg(b3 + 2);
    }
    // D2 is read before layer 2 of the next tile overwrites it
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (timeout) atomicOr(status, 1u);
  __syncthreads();
  if (w == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u)
                 : "memory");
}

// ---------------------------------------------------------------------------
// General training GEMM on the tensor cores: C[M][N] = A[M][K] B[N][K]^T, A
// and B BF16 and K-major (row pitch lda / ldb elements), N = 128 or 256, FP32
// accumulation in tensor memory.  One CTA of 4 warps per (128-row tile, K
// split): K chunks of 64 are staged by cp.async into two shared-memory
// stages in the canonical no-swizzle layout, one elected thread issues four
// M = 128, N, K = 16 MMAs per chunk and commits them to the stage's mbarrier,
// and the next chunk's copies overlap the current chunk's MMAs.  Epilogues:
//   kEpiF32       C[(split M + row) ldc + col] = acc (per-split partials when
//                 the K range is split; tc_split_sum adds them in split order)
//   kEpiBiasRelu  v = relu(acc + bias[col]) as BF16 into O[row][col] and,
//                 if OT, OT[col][row]
//   kEpiMask      v = acc where mask[row][col] > 0, else 0, into O and OT
// Rows of A at or beyond M are read as zero; K must be a multiple of 64 per
// split (the callers pad with zero columns).
// ---------------------------------------------------------------------------
enum { kEpiF32 = 0, kEpiBiasRelu = 1, kEpiMask = 2 };
constexpr int kGemmKc = 64;  // K per chunk

template <int N>
constexpr uint32_t idesc_n() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

// rows [r0, r0 + R) x columns [0, 64) of a K-major BF16 matrix (row pitch ld,
// columns already offset) into the canonical layout; rows at or beyond nrows
// are zero
__device__ __forceinline__ void load_chunk_async(unsigned char* dst, const uint16_t* __restrict__ src,
                                                 long long ld, long long r0, int R, long long nrows) {
  constexpr int kc8 = kGemmKc / 8;
  const int chunks = R * kc8;
  for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
    const int rr = c & 7, kc = (c >> 3) % kc8, rg = (c >> 3) / kc8;
    const long long r = r0 + rg * 8 + rr;
    const bool in = r < nrows;
    const uint16_t* g = src + (in ? r : 0) * ld + kc * 8;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst + (size_t)c * 16)),
                 "l"(g), "r"(in ? 16 : 0)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__global__ void __launch_bounds__(128, 1) tc_gemm_kernel(
    const uint16_t* __restrict__ A, long long lda, const uint16_t* __restrict__ B, long long ldb,
    long long M, int ksplit, int epi, float* __restrict__ C, long long ldc,
    uint16_t* __restrict__ O, long long ldo, uint16_t* __restrict__ OT, long long ldot,
    const float* __restrict__ bias, const uint16_t* __restrict__ mask, long long ldm,
    unsigned int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  constexpr uint32_t kA = TM * kGemmKc * 2, kB = N * kGemmKc * 2;  // bytes of one stage
  // stage s: A at dsm + s (kA + kB), B right after it
  uint64_t* mbar = reinterpret_cast<uint64_t*>(dsm + 2 * (kA + kB));  // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const long long r0 = (long long)blockIdx.x * TM;
  const long long k0 = (long long)blockIdx.y * ksplit;
  const int nch = ksplit / kGemmKc;

  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"((uint32_t)N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1u);
    mbar_init(&mbar[1], 1u);
    fence_mbar_init();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t lbo = 128u, sbo = (uint32_t)(kGemmKc / 8) * 128u;
  bool timeout = false;

  for (int i = 0; i < nch; ++i) {
    const int s = i & 1;
    // the MMAs of chunk i - 2 read this stage: wait for their commit
    if (i >= 2 && !mbar_wait(&mbar[s], (uint32_t)((i / 2 - 1) & 1))) timeout = true;
    const long long kk = k0 + (long long)i * kGemmKc;
    unsigned char* const sA = dsm + (size_t)s * (kA + kB);
    unsigned char* const sB = sA + kA;
    load_chunk_async(sA, A + kk, lda, r0, TM, M);
    load_chunk_async(sB, B + kk, ldb, 0, N, N);
    cp_async_wait_all();
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t ad = smem_desc(smem_u32(sA), lbo, sbo);
      const uint64_t bd = smem_desc(smem_u32(sB), lbo, sbo);
#pragma unroll
      for (int kb = 0; kb < kGemmKc / 16; ++kb) {
        const uint64_t adv = (uint64_t)((kb * 256) >> 4);
        const uint32_t acc = (i > 0 || kb > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad + adv), "l"(bd + adv), "r"(idesc_n<N>()), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&mbar[s]))
          : "memory");
    }
  }
  // the last commit covers every MMA issued before it
  if (nch > 0 && !mbar_wait(&mbar[(nch - 1) & 1], (uint32_t)(((nch - 1) / 2) & 1))) timeout = true;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // epilogue: warp w owns TMEM lanes (rows) 32 w .. 32 w + 31
  const long long row = r0 + 32 * w + lane;
  const bool live = row < M && nch > 0;
#pragma unroll 1
  for (int c0 = 0; c0 < N; c0 += 32) {
    uint32_t v[32];
    tmem_ld32(tmem + ((uint32_t)(32 * w) << 16) + (uint32_t)c0, v);
    if (epi == kEpiF32) {
      if (live) {
        float4* dst = reinterpret_cast<float4*>(C + ((long long)blockIdx.y * M + row) * ldc + c0);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          dst[q] = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                               __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
      }
      continue;
    }
    float f[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      float x = __uint_as_float(v[j]);
      if (epi == kEpiBiasRelu) {
        x = fmaxf(x + bias[c0 + j], 0.f);
      } else if (live) {
        const uint16_t mk = mask[row * ldm + c0 + j];
        if (!(__uint_as_float((uint32_t)mk << 16) > 0.f)) x = 0.f;
      }
      f[j] = x;
    }
    if (live) {
      uint32_t pk[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) pk[j] = bf16x2_bits(f[2 * j], f[2 * j + 1]);
      uint4* dst = reinterpret_cast<uint4*>(O + row * ldo + c0);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        dst[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
      if (OT) {
        // column c0 + j of the 32 rows of this warp: 64 contiguous bytes
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const __nv_bfloat16 b = __float2bfloat16_rn(f[j]);
          OT[(long long)(c0 + j) * ldot + row] = *reinterpret_cast<const uint16_t*>(&b);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  if (timeout) atomicOr(status, 1u);
  __syncthreads();
  if (w == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)N)
                 : "memory");
}

// G[i] = sum over splits s = 0, 1, ... of P[s][i], in that order
__global__ void tc_split_sum_kernel(const float* __restrict__ P, long long n, int splits,
                                    float* __restrict__ G) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int s = 0; s < splits; ++s) acc += P[(long long)s * n + i];
    G[i] = acc;
  }
}

}  // namespace

size_t tc_gemm_smem(int N) { return (size_t)2 * (TM + N) * kGemmKc * 2 + 16 + 16; }

// C[M][N] = A[M][K] B[N][K]^T on the tensor cores (see tc_gemm_kernel).
// epi 0: FP32 into C (row pitch ldc); with splits > 1 the K range is cut in
// `splits` parts whose partials go to `part` ([splits][M][N]) and are summed
// into C (pitch N) in split order, so the result does not depend on timing.
// epi 1 / 2: BF16 into O (and OT transposed, if not null).
int tc_gemm(const uint16_t* A, long long lda, const uint16_t* B, long long ldb, long long M, int N,
            long long K, int splits, int epi, float* C, long long ldc, float* part, uint16_t* O,
            long long ldo, uint16_t* OT, long long ldot, const float* bias, const uint16_t* mask,
            long long ldm, unsigned int* status, cudaStream_t st) {
  if (M <= 0) return QTV_OK;
  if (N != 128 && N != 256) return set_error(QTV_ERR_ARG, "tc_gemm: N = %d (128 or 256)", N);
  if (splits < 1 || K % ((long long)splits * kGemmKc) != 0)
    return set_error(QTV_ERR_ARG, "tc_gemm: K = %lld not a multiple of %d splits x %d", K, splits,
                     kGemmKc);
  if (splits > 1 && (epi != kEpiF32 || !part))
    return set_error(QTV_ERR_ARG, "tc_gemm: split K needs the FP32 epilogue and partials");
  static bool attr[2] = {false, false};
  const int which = N == 256 ? 1 : 0;
  const size_t smem = tc_gemm_smem(N);
  if (!attr[which]) {
    cudaError_t e = N == 256 ? cudaFuncSetAttribute(tc_gemm_kernel<256>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                             : cudaFuncSetAttribute(tc_gemm_kernel<128>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return check_cuda(e, "cudaFuncSetAttribute(tc_gemm)");
    attr[which] = true;
  }
  const dim3 grid((unsigned)((M + TM - 1) / TM), (unsigned)splits);
  const int ksplit = (int)(K / splits);
  float* Cout = splits > 1 ? part : C;
  const long long ldcc = splits > 1 ? N : ldc;
  if (N == 256)
    tc_gemm_kernel<256><<<grid, 128, smem, st>>>(A, lda, B, ldb, M, ksplit, epi, Cout, ldcc, O, ldo,
                                                 OT, ldot, bias, mask, ldm, status);
  else
    tc_gemm_kernel<128><<<grid, 128, smem, st>>>(A, lda, B, ldb, M, ksplit, epi, Cout, ldcc, O, ldo,
                                                 OT, ldot, bias, mask, ldm, status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return check_cuda(e, "tc_gemm_kernel launch");
  if (splits > 1) {
    const long long n = M * N;
    tc_split_sum_kernel<<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, st>>>(
        part, n, splits, C);
    e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(e, "tc_split_sum_kernel launch");
  }
  return QTV_OK;
}

size_t tc_dense_smem(int K) {
  return (size_t)(TN + TM) * K * 2 + 8 + 16 + TN * sizeof(float);
}

// out[M][256] = relu(A W^T + b) (BF16, row-major); A [M][K], W [256][K] BF16.
int tc_dense_relu(const uint16_t* A, long long M, int K, const uint16_t* W, const float* bias,
                  uint16_t* out, unsigned int* status, int num_sms, cudaStream_t st) {
  if (K != 128 && K != 256) return set_error(QTV_ERR_ARG, "tc_dense: K = %d (128 or 256)", K);
  if (M <= 0) return QTV_OK;
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(tc_dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024);
    if (e != cudaSuccess) return check_cuda(e, "cudaFuncSetAttribute(tc_dense)");
    attr = true;
  }
  const long long ntiles = (M + TM - 1) / TM;
  const int grid = (int)(ntiles < num_sms ? ntiles : num_sms);
  tc_dense_kernel<<<grid, 128, tc_dense_smem(K), st>>>(A, M, K, W, bias, out, status);
  return check_cuda(cudaGetLastError(), "tc_dense_kernel launch");
}

// Y[M][3] of the whole network on the tensor cores (see tc_mlp_kernel).
int tc_mlp_forward(const uint16_t* X, long long M, const uint16_t* W1, const uint16_t* W2,
                   const float* b1, const float* b2, const float* w3, const float* b3, float* Y,
                   unsigned int* status, int num_sms, cudaStream_t st) {
  if (M <= 0) return QTV_OK;
  const size_t smem = (size_t)kMlpSmemW1 + kMlpSmemW2 + kMlpSmemX + 32 + kMlpSmemPart;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tc_mlp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return check_cuda(e, "cudaFuncSetAttribute(tc_mlp)");
    attr = true;
  }
  const long long ntiles = (M + TM - 1) / TM;
  const int grid = (int)(ntiles < num_sms ? ntiles : num_sms);
  tc_mlp_kernel<<<grid, kMlpThreads, smem, st>>>(X, M, W1, W2, b1, b2, w3, b3, Y, status);
  return check_cuda(cudaGetLastError(), "tc_mlp_kernel launch");
}

}  // namespace qtv
