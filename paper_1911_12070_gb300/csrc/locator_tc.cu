// locator_tc.cu -- the learned locator's network on the 5th-generation tensor
// cores (tcgen05, accumulators in tensor memory): the training GEMM
// (tc_gemm_kernel) and the whole 128-256-256-3 network fused per 128-row tile
// (tc_mlp_kernel, warp-specialised; its design is described at its
// definition).
//
// Operands staged by threads are stored in the canonical K-major layout
// without swizzle: 8 x 8 core matrices of 128 contiguous bytes (8 rows of 16
// bytes), core matrix (r / 8, k / 8) at ((r / 8) (K / 8) + k / 8) 128 bytes,
// so the leading-dimension offset (next core matrix along K) is 128 bytes and
// the stride offset (next 8-row group) is 16 K bytes.  One elected thread
// issues the tcgen05.mma instructions and commits them to mbarriers; warps
// read their 32 TMEM lanes back with tcgen05.ld.  Accumulator columns are
// allocated once per CTA and freed before exit; every mbarrier wait is
// bounded and sets a status flag on timeout.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "qtv_internal.cuh"
#include "sweep_common.cuh"

namespace qtv {
namespace {

using namespace sweep;

constexpr int TM = 128;   // rows per tile (M of one instruction, TMEM lanes)

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

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// ---------------------------------------------------------------------------
// The whole network for 128-row tiles: Y[M][3] = W3 relu(W2 relu(W1 x + b1) +
// b2) + b3, one persistent CTA per SM.  W1 (64 KB) and W2 (128 KB) stay in
// shared memory in the no-swizzle layout above, with b1[0..127] and w3 rows
// 0 and 1; per tile the 128 X rows (32 KB) arrive by two tensor copies
// (cp.async.bulk.tensor, 64 columns each) in the 128-byte-swizzle K-major
// layout.  Tensor memory (512 columns) holds four 128-column quarters:
//   Q0, Q1  layer 1, hidden units 0..127 and 128..255 (FP32); epilogue 1
//           packs relu(. + b1) as BF16 pairs into the first 64 columns of
//           its own quarter (row = lane, two consecutive K values a column)
//   Q2, Q3  layer 2, outputs 0..127 and 128..255 (FP32)
// and every product is M = 128, N = 128, K = 16 so that the epilogues
// overlap the tensor cores.  Per tile t the issuing thread runs
//   L1(Q0) | L1(Q1) | L2(Q2, K 0..127) | L2(Q3, K 0..127) | L2(Q2, K 128..255)
//   L2(Q3, K 128..255)
// where each "|" waits for what the next products read or overwrite: this
// tile's X and layer 2 of t - 1 done with Q0; layer 2 of t - 1 done with Q1;
// epilogue 1 of Q0 and epilogue 2 of t - 1 done with Q2; epilogue 2 of t - 1
// done with Q3; epilogue 1 of Q1.  So epilogue 1 of Q0 runs beside L1(Q1),
// epilogue 1 of Q1 beside the first K half of layer 2, and epilogue 2 of t
// beside layer 1 and the first K half of layer 2 of t + 1; the tensor cores
// wait only for the part of epilogue 1 of Q0 that outlasts L1(Q1).
// Warp roles (14 warps; warp w reaches TMEM lanes 32 (w % 4) ..):
//   0-3    epilogue 1 (bias, ReLU, BF16 pairs) of Q0 and Q1
//   4-7    epilogue 2 of Q2 (hidden units 0..127): Y = partial + b3
//   8-11   epilogue 2 of Q3 (128..255): Y += partial, after warps 4-7
//   12     the issuing thread (tcgen05.mma, tcgen05.commit)
//   13     the X copies, once layer 1 of the previous tile has read X
// Epilogue 2 reads TMEM in the 16x256b shape, where a thread holds two
// adjacent hidden units of four rows, so each weight it loads serves four
// rows.  The epilogues use packed FP32 pair arithmetic (add/fma .f32x2) and
// round with cvt.rn.relu.bf16x2, which clamps at zero as relu followed by
// rounding does.  Every wait is bounded: a thread whose wait runs out stops
// waiting, the kernel finishes on junk in bounds and the status word is set.
// ---------------------------------------------------------------------------
constexpr uint32_t kMlpSmemW1 = 256 * 128 * 2, kMlpSmemW2 = 256 * 256 * 2, kMlpSmemX = 128 * 128 * 2;
constexpr int kMlpThreads = 448;  // 14 warps (roles above)
constexpr uint32_t kMlpBars = 14;  // 8-byte slots: 12 mbarriers, the TMEM base, padding
constexpr uint32_t kMlpSmemBias = (128 + 512) * sizeof(float);  // b1[0 .. 127], w3 rows 0 and 1
constexpr size_t kMlpSmem = (size_t)kMlpSmemW1 + kMlpSmemW2 + kMlpSmemX + 8 * kMlpBars + kMlpSmemBias;
static_assert(kMlpSmem <= 227 * 1024, "fused network shared memory");
// instruction descriptor of kind::f16 for M = 128, N = 128
constexpr uint32_t kIdesc128 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 3) << 17) |
                               ((uint32_t)(TM >> 4) << 24);

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

// as tmem_ld32 without the wait (complete with tmem_ld_wait before use)
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t* v) {
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
}
__device__ __forceinline__ void tmem_ld_wait() {
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

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mma_ss_i(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_ts_i(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// (o0, o1) = (a0 + b0, a1 + b1), one packed FP32 instruction, IEEE rounding per element
__device__ __forceinline__ void add_x2(float& o0, float& o1, float a0, float a1, float b0, float b1) {
  asm("{\n .reg .b64 a, b, d;\n mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %5};\n"
      " add.rn.f32x2 d, a, b;\n mov.b64 {%0, %1}, d;\n}"
      : "=f"(o0), "=f"(o1)
      : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// (d0, d1) += (a0 b0, a1 b1), fused per element
__device__ __forceinline__ void fma_x2(float& d0, float& d1, float a0, float a1, float b0, float b1) {
  asm("{\n .reg .b64 a, b, c;\n mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %5};\n"
      " mov.b64 c, {%0, %1};\n fma.rn.f32x2 c, a, b, c;\n mov.b64 {%0, %1}, c;\n}"
      : "+f"(d0), "+f"(d1)
      : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// BF16 pair (lo in the low half) of max(lo, 0), max(hi, 0), round to nearest even
__device__ __forceinline__ uint32_t relu_bf16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// epilogue 1 of one quarter for this warp's 32 rows: columns q .. q + 127 of
// tensor memory (q = the quarter's first column, lane offset included) hold
// layer-1 sums of 128 hidden units; relu(. + b) as BF16 pairs goes to
// columns q .. q + 63, one 32-column block at a time.  b comes from shared
// memory, or (global) from global memory, one coalesced load a block
// broadcast by shuffles.
__device__ __forceinline__ void mlp_epilogue1(uint32_t q, const float* __restrict__ sb, bool global) {
  uint32_t va[32], vb[32];
  tmem_ld32_nowait(q, va);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint32_t* v = (j & 1) ? vb : va;
    tmem_ld_wait();
    // block j + 1 (columns 32 j + 32 ..) is requested before block j is packed
    // into columns 16 j .. 16 j + 15, which blocks 0 .. j have already read
    if (j < 3) tmem_ld32_nowait(q + 32u * (j + 1), (j & 1) ? va : vb);
    uint32_t pk[16];
    // from global memory: lane i loads the bias of column 32 j + i (one
    // coalesced request) and shuffles broadcast it
    const float lb = global ? __ldg(sb + 32 * j + (threadIdx.x & 31)) : 0.f;
#pragma unroll
    for (int c = 0; c < 32; c += 4) {
      float4 b;
      if (global) {
        b.x = __shfl_sync(0xffffffffu, lb, c);
        b.y = __shfl_sync(0xffffffffu, lb, c + 1);
        b.z = __shfl_sync(0xffffffffu, lb, c + 2);
        b.w = __shfl_sync(0xffffffffu, lb, c + 3);
      } else {
        b = *reinterpret_cast<const float4*>(sb + 32 * j + c);
      }
      float a0, a1, a2, a3;
      add_x2(a0, a1, __uint_as_float(v[c]), __uint_as_float(v[c + 1]), b.x, b.y);
      add_x2(a2, a3, __uint_as_float(v[c + 2]), __uint_as_float(v[c + 3]), b.z, b.w);
      pk[c / 2] = relu_bf16x2(a0, a1);
      pk[c / 2 + 1] = relu_bf16x2(a2, a3);
    }
    tmem_st16(q + 16u * j, pk);
  }
}

// tcgen05.ld .16x256b.x4: 16 lanes from the lane of taddr, 32 columns.  For
// column group k (columns 8 k .. 8 k + 7) thread t receives v[4 k], v[4 k + 1]
// = lane t / 4, columns 8 k + 2 (t % 4) and the next one, and v[4 k + 2],
// v[4 k + 3] = lane t / 4 + 8, the same two columns
__device__ __forceinline__ void tmem_ld_16x256b_x4(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.16x256b.x4.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

// epilogue 2 of one quarter in the 16x256b fragment layout: each thread holds
// two adjacent hidden units of four rows (lanes t/4, t/4 + 8, t/4 + 16,
// t/4 + 24 of the warp's 32), so every weight it loads serves four rows.
// Columns q .. q + 127 hold layer-2 sums of the hidden units h0 .. h0 + 127;
// y[6 i + 2 o], y[6 i + 2 o + 1] are the even and odd partial sums of output
// o for row i.  w3 rows 0 and 1 come from shared memory (sw3), b2 and w3
// row 2 from global memory.
__device__ __forceinline__ void mlp_epilogue2(uint32_t q, const float* __restrict__ sw3,
                                              const float* __restrict__ b2,
                                              const float* __restrict__ w3, int h0, float* y) {
  const int cq = 2 * (threadIdx.x & 3);
  uint32_t va[32], vb[32];
  tmem_ld_16x256b_x4(q, va);
  tmem_ld_16x256b_x4(q + (16u << 16), va + 16);
#pragma unroll
  for (int cc = 0; cc < 4; ++cc) {
    uint32_t* v = (cc & 1) ? vb : va;
    tmem_ld_wait();
    if (cc < 3) {
      uint32_t* n = (cc & 1) ? va : vb;
      tmem_ld_16x256b_x4(q + 32u * (cc + 1), n);
      tmem_ld_16x256b_x4(q + (16u << 16) + 32u * (cc + 1), n + 16);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int h = h0 + 32 * cc + 8 * k + cq;
      const float2 bb = __ldg(reinterpret_cast<const float2*>(b2 + h));
      const float2 u0 = *reinterpret_cast<const float2*>(sw3 + h);
      const float2 u1 = *reinterpret_cast<const float2*>(sw3 + 256 + h);
      const float2 u2 = __ldg(reinterpret_cast<const float2*>(w3 + 512 + h));
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        // row i: lanes t/4 (i = 0), t/4 + 8 (1) of the first load, t/4 + 16 (2), t/4 + 24 (3)
        const uint32_t* p = v + (i >> 1) * 16 + 4 * k + 2 * (i & 1);
        float a0, a1;
        add_x2(a0, a1, __uint_as_float(p[0]), __uint_as_float(p[1]), bb.x, bb.y);
        a0 = fmaxf(a0, 0.f);
        a1 = fmaxf(a1, 0.f);
        fma_x2(y[6 * i], y[6 * i + 1], u0.x, u0.y, a0, a1);
        fma_x2(y[6 * i + 2], y[6 * i + 3], u1.x, u1.y, a0, a1);
        fma_x2(y[6 * i + 4], y[6 * i + 5], u2.x, u2.y, a0, a1);
      }
    }
  }
}

// the three outputs of row i of this thread's four (lane t/4 + 8 i of the
// warp's 32): the partial sums of the four threads t & ~3 .. t | 3 added
__device__ __forceinline__ void mlp_outputs(const float* y, float* out) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      float s = y[6 * i + 2 * o] + y[6 * i + 2 * o + 1];
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      out[3 * i + o] = s;
    }
  }
}

// rows y .. y + 127, columns x .. x + 63 of X by one tensor copy in the
// 128-byte swizzle: row r lands at 128 r bytes with its 16-byte pieces
// permuted by r % 8 (the K-major 128-byte-swizzle operand layout); completion
// counted in bytes on bar.  Rows past the matrix read as zero.
__device__ __forceinline__ void tma_load_x(void* dst, const CUtensorMap* map, int x, int y,
                                           uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__global__ void __launch_bounds__(kMlpThreads, 1) tc_mlp_kernel(
    const __grid_constant__ CUtensorMap xmap, long long M, const uint16_t* __restrict__ W1,
    const uint16_t* __restrict__ W2, const float* __restrict__ b1, const float* __restrict__ b2,
    const float* __restrict__ w3, const float* __restrict__ b3, float* __restrict__ Y,
    unsigned int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  unsigned char* sW1 = dsm;
  unsigned char* sW2 = dsm + kMlpSmemW1;
  unsigned char* sX = sW2 + kMlpSmemW2;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sX + kMlpSmemX);
  uint64_t* bar_l1a = bars + 0;   // layer 1 of the tile into Q0 done
  uint64_t* bar_l1b = bars + 1;   // layer 1 into Q1 done
  uint64_t* bar_k0 = bars + 2;    // layer 2 has read the first K half (Q0 free)
  uint64_t* bar_l2a = bars + 3;   // layer 2 into Q2 done
  uint64_t* bar_l2b = bars + 4;   // layer 2 into Q3 done (all of layer 2: Q1 free)
  uint64_t* bar_e1a = bars + 5;   // epilogue 1 wrote the BF16 pairs of Q0 (one arrival per warp)
  uint64_t* bar_e1b = bars + 6;   // epilogue 1 wrote those of Q1
  uint64_t* bar_e2a = bars + 7;   // epilogue 2 has read Q2
  uint64_t* bar_e2b = bars + 8;   // epilogue 2 has read Q3
  uint64_t* bar_xr = bars + 9;    // the next tile's X is in shared memory
  uint64_t* bar_ya = bars + 10;   // the first epilogue-2 group wrote its part of Y
  uint64_t* bar_fin = bars + 11;  // every product issued has completed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 12);
  float* sb1 = reinterpret_cast<float*>(bars + kMlpBars);  // b1[0 .. 127]
  float* sw3 = sb1 + 128;                                   // w3 rows 0 and 1
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int wq = w & 3;  // TMEM lane quarter (rows 32 wq .. 32 wq + 31)

  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < 5; ++i) mbar_init(bars + i, 1u);
    for (int i = 5; i < 9; ++i) mbar_init(bars + i, 4u);
    mbar_init(bar_xr, 1u);
    mbar_init(bar_ya, 4u);
    mbar_init(bar_fin, 1u);
    fence_mbar_init();
  }
  if (tid < 128) sb1[tid] = __ldg(b1 + tid);
  for (int i = tid; i < 512; i += kMlpThreads) sw3[i] = __ldg(w3 + i);
  load_canon(sW1, W1, 0, 256, 256, 128);
  load_canon(sW2, W2, 0, 256, 256, 256);
  const long long ntiles = (M + TM - 1) / TM;
  fence_proxy_async();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t lane_off = (uint32_t)(32 * wq) << 16;
  // a thread whose bounded wait has run out stops waiting: the rest of the
  // kernel runs unsynchronised (in bounds, on junk) and the status flags it
  bool tmo = false;
  auto wait = [&](uint64_t* bar, uint32_t parity) {
    if (!tmo && !mbar_wait(bar, parity)) tmo = true;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  };
  auto arrive = [&](uint64_t* bar) {  // one arrival per warp, after the warp's tensor-memory accesses
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncwarp();
    if (lane == 0) mbar_arrive(bar);
  };

  if (w == 12) {
    // the issuing thread: per tile 16 layer-1 and 32 layer-2 products (M = 128, N = 128, K = 16)
    if (lane == 0) {
      // X in two 128-byte-swizzled halves (K 0..63, 64..127) of 16 KB: 8-row
      // groups 1024 bytes apart; a K step of 16 moves the start by 32 bytes
      const uint64_t xdesc = smem_desc(smem_u32(sX), 16u, 1024u) | ((uint64_t)2 << 61);
      const uint64_t w1d0 = smem_desc(smem_u32(sW1), 128u, 16u * 128u);
      const uint64_t w1d1 = smem_desc(smem_u32(sW1 + 16 * 16 * 128), 128u, 16u * 128u);
      const uint64_t w2d0 = smem_desc(smem_u32(sW2), 128u, 32u * 128u);
      const uint64_t w2d1 = smem_desc(smem_u32(sW2 + 16 * 32 * 128), 128u, 32u * 128u);
      auto layer1 = [&](int n) {  // Q_n = X W1[128 n .. 128 n + 127]^T
        const uint64_t wd = n ? w1d1 : w1d0;
#pragma unroll
        for (int kb = 0; kb < 8; ++kb)
          mma_ss_i(tmem + 128u * n, xdesc + (uint64_t)((kb >> 2) * 1024 + (kb & 3) * 2),
                   wd + (uint64_t)(kb * 16),
                   kIdesc128, kb > 0 ? 1u : 0u);
      };
      auto layer2 = [&](int n, int k) {  // Q_{2+n} += A1 (K half k, in Q_k) W2[128 n .., 128 k ..]^T
        const uint64_t wd = (n ? w2d1 : w2d0) + (uint64_t)(k * 128);
#pragma unroll
        for (int kb = 0; kb < 8; ++kb)
          mma_ts_i(tmem + 256u + 128u * n, tmem + 128u * k + 8u * kb, wd + (uint64_t)(kb * 16),
                   kIdesc128, (k > 0 || kb > 0) ? 1u : 0u);
      };
      uint32_t ph = 0;
      int it = 0;
      for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ph ^= 1u, ++it) {
        wait(bar_xr, ph);                    // this tile's X
        if (it > 0) wait(bar_k0, ph ^ 1u);  // the previous tile's layer 2 done with Q0
        layer1(0);
        mma_commit(bar_l1a);
        if (it > 0) wait(bar_l2b, ph ^ 1u);  // ... and with Q1
        layer1(1);
        mma_commit(bar_l1b);
        wait(bar_e1a, ph);
        if (it > 0) wait(bar_e2a, ph ^ 1u);  // the previous tile's epilogue 2 has read Q2
        layer2(0, 0);
        if (it > 0) wait(bar_e2b, ph ^ 1u);  // ... and Q3
        layer2(1, 0);
        mma_commit(bar_k0);
        wait(bar_e1b, ph);
        layer2(0, 1);
        mma_commit(bar_l2a);
        layer2(1, 1);
        mma_commit(bar_l2b);
      }
      // every product has completed before the columns are freed
      mma_commit(bar_fin);
      if (!mbar_wait(bar_fin, 0u)) tmo = true;
    }
  } else if (w == 13) {
    // the X copies: two tensor copies of 128 rows x 64 columns per tile,
    // issued once both layer-1 halves of the previous tile have read X
    if (lane == 0) {
      uint32_t ph = 0;
      int it = 0;
      for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ph ^= 1u, ++it) {
        if (it > 0) wait(bar_l1b, ph ^ 1u);
        mbar_arrive_expect_tx(bar_xr, kMlpSmemX);
        tma_load_x(sX, &xmap, 0, (int)(tile * TM), bar_xr);
        tma_load_x(sX + kMlpSmemX / 2, &xmap, 64, (int)(tile * TM), bar_xr);
      }
    }
  } else if (w < 4) {
    // epilogue 1 of both halves
    uint32_t ph = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ph ^= 1u) {
      wait(bar_l1a, ph);
      __syncwarp();
      mlp_epilogue1(tmem + lane_off, sb1, false);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      arrive(bar_e1a);
      wait(bar_l1b, ph);
      __syncwarp();
      mlp_epilogue1(tmem + lane_off + 128u, b1 + 128, true);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      arrive(bar_e1b);
    }
  } else {
    // epilogue 2: warps 4-7 the hidden units 0..127 (Q2), which write
    // Y = their partial sums + b3; warps 8-11 those of 128..255 (Q3), which
    // add theirs once the first group's are in Y
    const bool upper = w >= 8;
    uint32_t ph = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ph ^= 1u) {
      // this thread writes row lane / 4 + 8 (lane % 4) of the warp's 32
      const long long row = tile * TM + 32 * wq + (lane >> 2) + 8 * (lane & 3);
      float y[24];
#pragma unroll
      for (int i = 0; i < 24; ++i) y[i] = 0.f;
      wait(upper ? bar_l2b : bar_l2a, ph);
      __syncwarp();
      mlp_epilogue2(tmem + lane_off + (upper ? 384u : 256u), sw3, b2, w3, upper ? 128 : 0, y);
      float out[12];
      mlp_outputs(y, out);
      const int k = lane & 3;
      float r[3];
#pragma unroll
      for (int o = 0; o < 3; ++o)  // row k of the four (selects, no indexed register array)
        r[o] = k == 0 ? out[o] : k == 1 ? out[3 + o] : k == 2 ? out[6 + o] : out[9 + o];
      if (!upper) {
        arrive(bar_e2a);  // Q2 may be overwritten
        if (row < M) {
          Y[3 * row] = r[0] + __ldg(b3);
          Y[3 * row + 1] = r[1] + __ldg(b3 + 1);
          Y[3 * row + 2] = r[2] + __ldg(b3 + 2);
        }
        __threadfence_block();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar_ya);
      } else {
        wait(bar_ya, ph);  // before Q3 is released: keeps the two groups one tile apart at most
        arrive(bar_e2b);
        if (row < M) {
          Y[3 * row] += r[0];
          Y[3 * row + 1] += r[1];
          Y[3 * row + 2] += r[2];
        }
      }
    }
  }
  if (tmo) atomicOr(status, 1u);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
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

// Y[M][3] of the whole network on the tensor cores (see tc_mlp_kernel).
int tc_mlp_forward(const uint16_t* X, long long M, const uint16_t* W1, const uint16_t* W2,
                   const float* b1, const float* b2, const float* w3, const float* b3, float* Y,
                   unsigned int* status, int num_sms, cudaStream_t st) {
  if (M <= 0) return QTV_OK;
  // 16-byte aligned operands (X for the tensor copies, b2 and w3 read as
  // 8-byte pairs); tile rows are 32-bit tensor coordinates
  if (((reinterpret_cast<uintptr_t>(b1) | reinterpret_cast<uintptr_t>(b2) |
        reinterpret_cast<uintptr_t>(w3) | reinterpret_cast<uintptr_t>(X)) & 15u) ||
      M >= (1ll << 31))
    return set_error(QTV_ERR_ARG, "fused network: misaligned operand or too many rows");
  const size_t smem = kMlpSmem;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tc_mlp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return check_cuda(e, "cudaFuncSetAttribute(tc_mlp)");
    attr = true;
  }
  const long long ntiles = (M + TM - 1) / TM;
  const int grid = (int)(ntiles < num_sms ? ntiles : num_sms);
  // X as a 2-D BF16 tensor (128 columns, M rows, 256-byte rows); boxes of
  // 64 columns x 128 rows, 128-byte swizzle, rows past M read as zero
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return check_cuda(e != cudaSuccess ? e : cudaErrorNotSupported, "cuTensorMapEncodeTiled");
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  CUtensorMap xmap;
  const cuuint64_t dims[2] = {128, (cuuint64_t)M};
  const cuuint64_t strides[1] = {256};
  const cuuint32_t box[2] = {64, (cuuint32_t)TM};
  const cuuint32_t estr[2] = {1, 1};
  if (encode(&xmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t*>(X), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return set_error(QTV_ERR_ARG, "tensor map of the network input");
  tc_mlp_kernel<<<grid, kMlpThreads, smem, st>>>(xmap, M, W1, W2, b1, b2, w3, b3, Y, status);
  return check_cuda(cudaGetLastError(), "tc_mlp_kernel launch");
}

}  // namespace qtv
