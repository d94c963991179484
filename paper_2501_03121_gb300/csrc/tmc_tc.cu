// Tensor-matrix contraction (TMC, Section 1) on the tensor cores, for BF16
// storage (every mode) and FP32 storage (the last mode; see the FP32 section
// below).  With A read as u x n_k x v (Section 3), every slab i is a matrix
// product:
//     Y[i][r][l] = alpha * scale * sum_j A[i][j][l] X[r][j] + beta * Y[i][r][l],
// X the R x n_k FP32 matrix.  Along the last mode (v = 1) the rows of A are
// the M dimension and the contracted index is contiguous (K-major tiles);
// along any other mode the v columns of a slab are the M dimension and are
// contiguous (MN-major tiles).
//
// X is split on the device into three BF16 pieces, X = X0 + X1 + X2 to
// binary32 precision (each piece the BF16 rounding of what the previous ones
// left).  A product of two BF16 values is exact in FP32, so the tensor cores
// form A[i][j] X_p[r][j] exactly and accumulate in FP32 in tensor memory:
// the result carries FP32 accumulation error only, like the CUDA-core path.
//
// Dataflow (one CTA per 128 outputs: rows of A, or columns of one slab):
//   - a producer thread brings, per block of 64 codes along n_k, the 128 x 64
//     tile of A (one box, or two 64 x 64 boxes along v for MN-major tiles)
//     and the three R_p x 64 tiles of X pieces into one stage of a
//     shared-memory ring with TMA (2-D tensor maps, 128-byte swizzle; rows
//     past u and codes past n_k are filled with zeros);
//   - one thread issues the MMAs (tcgen05.mma kind::f16, M = 128, K = 16 per
//     instruction; the three piece tiles are read as one tile of N = 3 R_p
//     rows, R_p = R rounded up to 16, so each K step is one MMA and each
//     piece accumulates in its own group of R_p columns) into FP32
//     accumulators in tensor memory, and returns the stage to the producer
//     with tcgen05.commit on its "empty" barrier;
//   - after the last block the four warps read the 128 x 3 R_p accumulators
//     back with tcgen05.ld (warp w owns rows 32w .. 32w + 31), add the three
//     groups (smallest first) and write Y.
// Every barrier wait is bounded in time; a wait that gives up records a code
// in a device word (read by tvc_device_error) and the CTA still releases its
// tensor memory.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "tma.cuh"

namespace tvcg {

namespace {

__device__ int g_tmc_tc_error = 0;

constexpr int kTcThreads = 128;
constexpr int kTcRows = 128;      // M: rows of A per CTA (one TMEM lane each)
constexpr int kTcK = 64;          // codes per stage along n_k: one 128-byte swizzle row
constexpr int kTileA = kTcRows * kTcK * 2;  // 16 KB

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Whole-warp allocation of `ncols` tensor-memory columns (a power of two >= 32);
// the base address is written to *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D (tensor memory) [+]= A (shared, descriptor) * B (shared, descriptor)^T.
__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrives on `bar` once every MMA this thread issued before has completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 tensor-memory lanes (one
// lane per thread), waited for before returning.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int q = 0; q < 16; q++) v[q] = __uint_as_float(r[q]);
}

// Shared-memory matrix descriptor of a K-major tile whose rows are 128 bytes
// (64 BF16) laid out by TMA with the 128-byte swizzle: start address, leading
// byte offset (unused for swizzled K-major tiles, 16), stride byte offset
// 1024 (8 rows of 128 bytes), descriptor version 1, swizzle mode 128 bytes.
__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// The same for an MN-major tile (M contiguous): 64-element (128-byte) rows
// along M, one row per K index, 8-row groups of 1024 bytes along K (stride
// byte offset), and the next 64 elements of M `atom_bytes` further (leading
// byte offset).
__device__ __forceinline__ uint64_t sw128_mnmajor_desc(uint32_t saddr, uint32_t atom_bytes) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((atom_bytes >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, B
// K-major, A K-major or (mn_a) MN-major, N = n columns, M = 128 rows.
__host__ __device__ constexpr uint32_t bf16_idesc(uint32_t n, bool mn_a = false) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((mn_a ? 1u : 0u) << 15) | ((n >> 3) << 17) |
         ((uint32_t)(kTcRows >> 4) << 24);
}

// ----------------------------------------------------------------- kernels

// X (R x nk FP32) -> three BF16 pieces, pieces[p][r][j] for r < Rp, j < nkp,
// zero outside R x nk: X0 = bf16(x), X1 = bf16(x - X0), X2 = bf16(x - X0 - X1)
// (the differences are exact in FP32).
// jscale (nullable): per-j factors folded into X first (mode 0 of narrow
// storage, where the slab scale runs along the contracted index).
__global__ void tmc_tc_split_x_kernel(const float* __restrict__ X, uint16_t* __restrict__ pieces, int64_t R,
                                      int64_t nk, int64_t Rp, int64_t nkp, const float* __restrict__ jscale) {
  const int64_t n = Rp * nkp;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = o / nkp, j = o - r * nkp;
    float x = (r < R && j < nk) ? X[r * nk + j] : 0.0f;
    if (jscale != nullptr && j < nk) x = __fmul_rn(x, jscale[j]);
    const __nv_bfloat16 h0 = __float2bfloat16_rn(x);
    const float rem1 = __fsub_rn(x, __bfloat162float(h0));
    const __nv_bfloat16 h1 = __float2bfloat16_rn(rem1);
    const float rem2 = __fsub_rn(rem1, __bfloat162float(h1));
    const __nv_bfloat16 h2 = __float2bfloat16_rn(rem2);
    pieces[o] = __bfloat16_as_ushort(h0);
    pieces[n + o] = __bfloat16_as_ushort(h1);
    pieces[2 * n + o] = __bfloat16_as_ushort(h2);
  }
}

struct TcArgs {
  float* Y;
  const float* scales;  // per slab (row i of the u x n_k x v view), nullable
  int64_t u, R, upi0, v, vt;  // vt: tiles of 128 along v (1 when v == 1)
  const float* A;             // FP32 slabs (v > 1), read by the converter warps
  int64_t nk;
  int Rp, nkb, stages, ncols;
  uint32_t stage_bytes;
  float alpha, beta;
};

// One CTA: 128 outputs of Y.  MN == false (v == 1): rows m0 .. m0 + 127 of
// the u x n_k matrix A (K-major tiles).  MN == true (v > 1): slab i of A, an
// n_k x v matrix, and columns l0 .. l0 + 127 of it (MN-major tiles: two
// 64-wide boxes per stage, 8 KB apart).  Warp 0 lane 0 produces (TMA), warp 1
// lane 0 issues the MMAs, all four warps run the epilogue.
template <bool MN>
__global__ void __launch_bounds__(kTcThreads) tmc_tc_kernel(const __grid_constant__ CUtensorMap mapA,
                                                           const __grid_constant__ CUtensorMap mapX,
                                                           const TcArgs a) {
  extern __shared__ unsigned char smraw[];
  // stages start at a 1024-byte boundary (the 128-byte swizzle atom)
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smraw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int S = a.stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + (size_t)S * a.stage_bytes);
  uint64_t* empty = full + S;
  uint64_t* done = empty + S;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tile_i = MN ? (int64_t)blockIdx.x / a.vt : 0;               // slab (MN)
  const int64_t m0 = MN ? ((int64_t)blockIdx.x % a.vt) * kTcRows : (int64_t)blockIdx.x * kTcRows;
  const uint32_t tile_x = (uint32_t)a.Rp * 128u;  // bytes of one piece's R_p x 64 tile

  if (threadIdx.x == 0) {
    for (int q = 0; q < S; q++) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    mbar_init(done, 1);
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, (uint32_t)a.ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  __shared__ int mma_ok;  // every MMA of the tile was issued

  if (warp == 0 && lane == 0) {
    // producer
    const uint32_t bytes = (uint32_t)kTileA + 3u * tile_x;
    int kb = 0;
    for (; kb < a.nkb; kb++) {
      const int st = kb % S;
      if (kb >= S && !mbar_wait(&empty[st], (uint32_t)((kb / S) - 1) & 1u, &g_tmc_tc_error, 1)) break;
      unsigned char* base = sm + (size_t)st * a.stage_bytes;
      mbar_arrive_expect_tx(&full[st], bytes);
      if constexpr (MN) {
        tma_load_3d(base, &mapA, (int)m0, kb * kTcK, (int)tile_i, &full[st]);
        tma_load_3d(base + kTileA / 2, &mapA, (int)m0 + 64, kb * kTcK, (int)tile_i, &full[st]);
      } else {
        tma_load_2d(base, &mapA, kb * kTcK, (int)m0, &full[st]);
      }
      for (int p = 0; p < 3; p++)
        tma_load_2d(base + kTileA + p * tile_x, &mapX, kb * kTcK, p * a.Rp, &full[st]);
    }
    // never leave with copies in flight
    for (int q = 0; q < S && q < kb; q++) {
      const int kk = kb - 1 - q;
      mbar_wait(&full[kk % S], (uint32_t)(kk / S) & 1u, &g_tmc_tc_error, 3, 400000000LL);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = bf16_idesc(3u * (uint32_t)a.Rp, MN);
    int kb = 0;
    for (; kb < a.nkb; kb++) {
      const int st = kb % S;
      if (!mbar_wait(&full[st], (uint32_t)(kb / S) & 1u, &g_tmc_tc_error, 2)) break;
      tc_fence_after();
      const uint32_t abase = smem_u32(sm + (size_t)st * a.stage_bytes);
      // the three piece tiles are one K-major tile of 3 R_p rows: one MMA per
      // K step, the pieces' products in column groups [p R_p, (p + 1) R_p)
#pragma unroll
      for (int kk = 0; kk < kTcK / 16; kk++) {
        // K step kk: 32 bytes along a K-major row, or 16 rows (2 groups of
        // 8 x 128 bytes) of an MN-major tile
        const uint64_t ad = MN ? sw128_mnmajor_desc(abase + kk * 2048u, (uint32_t)kTileA / 2)
                               : sw128_kmajor_desc(abase + kk * 32u);
        const uint64_t bd = sw128_kmajor_desc(abase + (uint32_t)kTileA + kk * 32u);
        tc_mma_bf16(tmem, ad, bd, idesc, (kb | kk) != 0 ? 1u : 0u);
      }
      tc_commit(&empty[st]);  // the stage is free once these MMAs have read it
    }
    mma_ok = (kb == a.nkb) ? 1 : 0;
    tc_commit(done);
  }
  __syncwarp();
  __syncthreads();  // mma_ok is visible; the producer has drained its copies

  // epilogue: warp w reads tensor-memory lanes 32w .. 32w + 31 (rows of Y)
  const bool ok = mbar_wait(done, 0u, &g_tmc_tc_error, 4) && mma_ok != 0;
  tc_fence_after();
  // output row of this thread: i (v == 1) or column l of slab tile_i
  const int64_t row = m0 + warp * 32 + lane;
  const int64_t i = MN ? tile_i : row;
  const bool live = MN ? row < a.v : row < a.u;
  const float sc = (a.scales != nullptr && live) ? a.scales[i / a.upi0] : 1.0f;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  for (int c0 = 0; c0 < a.Rp; c0 += 16) {
    float v0[16], v1[16], v2[16];
    tmem_ld16(trow + (uint32_t)c0, v0);
    tmem_ld16(trow + (uint32_t)(a.Rp + c0), v1);
    tmem_ld16(trow + (uint32_t)(2 * a.Rp + c0), v2);
    if (ok && live) {
#pragma unroll
      for (int q = 0; q < 16; q++) {
        const int64_t r = c0 + q;
        if (r < a.R) {
          const float acc = __fadd_rn(__fadd_rn(v2[q], v1[q]), v0[q]);  // smallest pieces first
          float out = __fmul_rn(__fmul_rn(acc, sc), a.alpha);
          const int64_t o = MN ? (i * a.R + r) * a.v + row : i * a.R + r;  // Y[i][r][l] / Y[i][r]
          if (a.beta != 0.0f) out = __fmaf_rn(a.beta, a.Y[o], out);
          a.Y[o] = out;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)a.ncols);
  }
}

// ------------------------------------------------------------ FP32 storage
//
// kind::tf32 reads an FP32 container through its sign, exponent and top 10
// fraction bits.  A (FP32, from TMA) serves as its own high part; four
// converter warps write A_lo = A - trunc(A) (trunc keeps those 19 bits; the
// difference is exact) into a second tile of the stage, elementwise at the
// same swizzled offsets.  X is split likewise: X_hi = trunc(X), X_lo = X -
// X_hi.  Two MMAs per K step of 8: A [X_hi; X_lo] (N = 2 R_p, accumulator
// groups 0 and 1) and A_lo X_hi (N = R_p, into group 1); the products
// dropped (A_lo X_lo, the bits of A_lo and X_lo beyond the container's 11)
// are below 2^-20 of |A X|.  Y = group 1 + group 0.

constexpr int kTcKf = 32;                      // FP32 per stage along n_k: one 128-byte row
constexpr int kTileAf = kTcRows * kTcKf * 4;  // 16 KB

constexpr uint32_t kTf32Mask = 0xFFFFE000u;
// Slab (MN) kernel: shared-memory stages, and stages of each converter
// thread's column in flight (1024^3 FP32 mode 1, R = 16, TB/s: 3 in flight /
// 2 stages 4.89, 4 / 2 4.84, 3 / 3 4.45, 2 / 3 4.29, 1 / 2 3.70; R = 32 needs
// the 2 stages to keep two CTAs per SM)
constexpr int kStagesMN = 2;
constexpr int kAheadMN = 3;

__global__ void tmc_tc_split_x_f32_kernel(const float* __restrict__ X, float* __restrict__ pieces, int64_t R,
                                          int64_t nk, int64_t Rp, int64_t nkp) {
  const int64_t n = Rp * nkp;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = o / nkp, j = o - r * nkp;
    const float x = (r < R && j < nk) ? X[r * nk + j] : 0.0f;
    const float hi = __uint_as_float(__float_as_uint(x) & kTf32Mask);
    pieces[o] = hi;
    pieces[n + o] = __fsub_rn(x, hi);
  }
}

__host__ __device__ constexpr uint32_t tf32_idesc(uint32_t n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((n >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}

// Component q (a compile-time constant after unrolling) of a float4.
__device__ __forceinline__ float f4_at(const float4& f, int q) {
  return q == 0 ? f.x : q == 1 ? f.y : q == 2 ? f.z : f.w;
}

// Two 4 x 4 blocks of a slab for one stage starting at row k0: rows
// k0 + 4 c_r + i (i = 0..3) of four adjacent columns, row stride v; zero past
// n_k or outside the slab.  Streamed: each value is read once.
__device__ __forceinline__ void tc_load_blocks(float4 (&d)[2][4], const float* src, int64_t k0, int c0, int c1,
                                               int64_t nk, int64_t v, bool cin) {
#pragma unroll
  for (int r = 0; r < 2; r++) {
    const int64_t k = k0 + 4 * (r ? c1 : c0);
    const float* p = src + k * v;
#pragma unroll
    for (int i = 0; i < 4; i++) {
      d[r][i] = (cin && k + i < nk) ? __ldcs(reinterpret_cast<const float4*>(p)) : make_float4(0.f, 0.f, 0.f, 0.f);
      p += v;
    }
  }
}

constexpr int kTcThreadsF = 192;  // producer warp, MMA warp, four converter / epilogue warps

// FP32 storage.  MN == false: rows m0 .. m0 + 127 of the u x n_k matrix A
// (the last mode, K-major tiles; the TMA tile serves as the high part).
// MN == true: columns l0 .. l0 + 127 of slab i.  The tf32 MMAs take K-major
// operands, so the converter warps read the slab themselves, one column per
// thread (each k a coalesced 128-byte load of the warp, one stage ahead in
// registers), and write the high and low parts as K-major tiles: shared
// memory sees no copy of A that is only read back to be transposed.
template <bool MN>
__global__ void __launch_bounds__(kTcThreadsF) tmc_tc_f32_kernel(const __grid_constant__ CUtensorMap mapA,
                                                                const __grid_constant__ CUtensorMap mapX,
                                                                const TcArgs a) {
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smraw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int S = a.stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + (size_t)S * a.stage_bytes);
  uint64_t* conv = full + S;
  uint64_t* empty = conv + S;
  uint64_t* done = empty + S;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ int mma_ok;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tile_i = MN ? (int64_t)blockIdx.x / a.vt : 0;
  const int64_t m0 = MN ? ((int64_t)blockIdx.x % a.vt) * kTcRows : (int64_t)blockIdx.x * kTcRows;
  const uint32_t tile_x = 2u * (uint32_t)a.Rp * 128u;  // X_hi and X_lo rows, 128 bytes each

  if (threadIdx.x == 0) {
    for (int q = 0; q < S; q++) {
      mbar_init(&full[q], 1);
      mbar_init(&conv[q], 128);
      mbar_init(&empty[q], 1);
    }
    mbar_init(done, 1);
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, (uint32_t)a.ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // producer
      const uint32_t bytes = (MN ? 0u : (uint32_t)kTileAf) + tile_x;
      int kb = 0;
      for (; kb < a.nkb; kb++) {
        const int st = kb % S;
        if (kb >= S && !mbar_wait(&empty[st], (uint32_t)((kb / S) - 1) & 1u, &g_tmc_tc_error, 1)) break;
        unsigned char* base = sm + (size_t)st * a.stage_bytes;
        mbar_arrive_expect_tx(&full[st], bytes);
        if constexpr (!MN) tma_load_2d(base, &mapA, kb * kTcKf, (int)m0, &full[st]);
        tma_load_2d(base + 2 * kTileAf, &mapX, kb * kTcKf, 0, &full[st]);
      }
      for (int q = 0; q < S && q < kb; q++) {
        const int kk = kb - 1 - q;
        mbar_wait(&full[kk % S], (uint32_t)(kk / S) & 1u, &g_tmc_tc_error, 3, 400000000LL);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      const uint32_t id2 = tf32_idesc(2u * (uint32_t)a.Rp), id1 = tf32_idesc((uint32_t)a.Rp);
      int kb = 0;
      for (; kb < a.nkb; kb++) {
        const int st = kb % S;
        if (!mbar_wait(&conv[st], (uint32_t)(kb / S) & 1u, &g_tmc_tc_error, 2)) break;
        tc_fence_after();
        const uint32_t base = smem_u32(sm + (size_t)st * a.stage_bytes);
#pragma unroll
        for (int kk = 0; kk < kTcKf / 8; kk++) {
          // K-major tiles: high part, low part, X; K step kk is 32 bytes
          // along the rows
          const uint64_t ahi = sw128_kmajor_desc(base + kk * 32u);
          const uint64_t alo = sw128_kmajor_desc(base + (uint32_t)kTileAf + kk * 32u);
          const uint64_t bx = sw128_kmajor_desc(base + 2u * (uint32_t)kTileAf + kk * 32u);
          tc_mma_tf32(tmem, ahi, bx, id2, (kb | kk) != 0 ? 1u : 0u);   // groups 0, 1
          tc_mma_tf32(tmem + (uint32_t)a.Rp, alo, bx, id1, 1u);          // A_lo X_hi into group 1
        }
        tc_commit(&empty[st]);
      }
      mma_ok = (kb == a.nkb) ? 1 : 0;
      tc_commit(done);
    }
  } else {
    const int t = threadIdx.x - 64;
    if constexpr (MN) {
      // thread t = 32 w + l: columns l0 + 4 l .. + 3 of slab i (rows 4 l ..
      // 4 l + 3 of the K-major tiles) and, per stage, the 4-row blocks
      // c_r = (2 w + r + l / 2) mod 8, r = 0, 1 (rows 4 c_r .. 4 c_r + 3 of the
      // stage): 16-byte loads, a 4 x 4 transpose in registers, and 16-byte
      // stores whose swizzled chunks c_r ^ (row % 8) differ across each 8 lanes.
      // A ring of kAheadMN stages in registers keeps that many in flight.
      const int w = t >> 5, l = t & 31;
      const int64_t col = m0 + 4 * l;
      const bool cin = col < a.v;  // v % 4 == 0: all four columns or none
      const float* src = a.A + tile_i * a.nk * a.v + (cin ? col : 0);
      const int c0 = (2 * w + (l >> 1)) & 7, c1 = (c0 + 1) & 7;
      float4 buf[kAheadMN][2][4];
#pragma unroll
      for (int j = 0; j < kAheadMN; j++)
        if (j < a.nkb) tc_load_blocks(buf[j], src, (int64_t)j * kTcKf, c0, c1, a.nk, a.v, cin);
      bool ok = true;
      for (int kb0 = 0; ok && kb0 < a.nkb; kb0 += kAheadMN) {
#pragma unroll
        for (int j = 0; j < kAheadMN; j++) {
          const int kb = kb0 + j, st = kb % S;
          if (!ok || kb >= a.nkb) break;
          if (kb >= S && !mbar_wait(&empty[st], (uint32_t)((kb / S) - 1) & 1u, &g_tmc_tc_error, 5)) {
            ok = false;
            break;
          }
          unsigned char* base = sm + (size_t)st * a.stage_bytes;
#pragma unroll
          for (int r = 0; r < 2; r++) {
            const int c = r ? c1 : c0;
#pragma unroll
            for (int q = 0; q < 4; q++) {
              const float e0 = f4_at(buf[j][r][0], q), e1 = f4_at(buf[j][r][1], q);
              const float e2 = f4_at(buf[j][r][2], q), e3 = f4_at(buf[j][r][3], q);
              float4 hi, lo;
              hi.x = __uint_as_float(__float_as_uint(e0) & kTf32Mask);
              hi.y = __uint_as_float(__float_as_uint(e1) & kTf32Mask);
              hi.z = __uint_as_float(__float_as_uint(e2) & kTf32Mask);
              hi.w = __uint_as_float(__float_as_uint(e3) & kTf32Mask);
              lo.x = __fsub_rn(e0, hi.x);
              lo.y = __fsub_rn(e1, hi.y);
              lo.z = __fsub_rn(e2, hi.z);
              lo.w = __fsub_rn(e3, hi.w);
              const int m = 4 * l + q;
              const int dst = m * 128 + ((c ^ (m & 7)) << 4);  // 128-byte swizzle
              *reinterpret_cast<float4*>(base + dst) = hi;
              *reinterpret_cast<float4*>(base + kTileAf + dst) = lo;
            }
          }
          if (kb + kAheadMN < a.nkb)
            tc_load_blocks(buf[j], src, (int64_t)(kb + kAheadMN) * kTcKf, c0, c1, a.nk, a.v, cin);
          if (!mbar_wait(&full[st], (uint32_t)(kb / S) & 1u, &g_tmc_tc_error, 5)) {  // X of the stage
            ok = false;
            break;
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
          mbar_arrive(&conv[st]);
        }
      }
    } else {
      // A_lo of every stage, 128 threads x 8 chunks of 16 bytes
      for (int kb = 0; kb < a.nkb; kb++) {
        const int st = kb % S;
        if (!mbar_wait(&full[st], (uint32_t)(kb / S) & 1u, &g_tmc_tc_error, 5)) break;
        unsigned char* base = sm + (size_t)st * a.stage_bytes;
#pragma unroll
        for (int c = 0; c < kTileAf / 16 / 128; c++) {
          const int off = (c * 128 + t) * 16;
          const float4 v = *reinterpret_cast<const float4*>(base + off);
          float4 lo;
          lo.x = __fsub_rn(v.x, __uint_as_float(__float_as_uint(v.x) & kTf32Mask));
          lo.y = __fsub_rn(v.y, __uint_as_float(__float_as_uint(v.y) & kTf32Mask));
          lo.z = __fsub_rn(v.z, __uint_as_float(__float_as_uint(v.z) & kTf32Mask));
          lo.w = __fsub_rn(v.w, __uint_as_float(__float_as_uint(v.w) & kTf32Mask));
          *reinterpret_cast<float4*>(base + kTileAf + off) = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
        mbar_arrive(&conv[st]);
      }
    }
  }
  __syncwarp();
  __syncthreads();

  if (warp >= 2) {  // epilogue: warp w reads tensor-memory lanes 32 (w % 4) ..
    const int q4 = warp & 3;
    const bool ok = mbar_wait(done, 0u, &g_tmc_tc_error, 4) && mma_ok != 0;
    tc_fence_after();
    const int64_t row = m0 + q4 * 32 + lane;
    const int64_t i = MN ? tile_i : row;
    const bool live = MN ? row < a.v : row < a.u;
    const uint32_t trow = tmem + ((uint32_t)(q4 * 32) << 16);
    for (int c0 = 0; c0 < a.Rp; c0 += 16) {
      float g0[16], g1[16];
      tmem_ld16(trow + (uint32_t)c0, g0);
      tmem_ld16(trow + (uint32_t)(a.Rp + c0), g1);
      if (ok && live) {
#pragma unroll
        for (int q = 0; q < 16; q++) {
          const int64_t r = c0 + q;
          if (r < a.R) {
            float out = __fmul_rn(__fadd_rn(g1[q], g0[q]), a.alpha);
            const int64_t o = MN ? (i * a.R + r) * a.v + row : i * a.R + r;
            if (a.beta != 0.0f) out = __fmaf_rn(a.beta, a.Y[o], out);
            a.Y[o] = out;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)a.ncols);
  }
}

}  // namespace
}  // namespace tvcg

namespace tvcg {

EncodeTiledFn encode_tiled() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

namespace {

// Row-major rows x cols BF16 matrix (row stride `stride` elements) read in
// boxes of box_rows x 64 with the 128-byte swizzle; zero fill outside.
bool encode_bf16_rows(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int64_t stride, int box_rows) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)stride * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The slabs of a u x n_k x v BF16 tensor (v contiguous, v > 1) read in
// boxes of 64 (along v) x 64 (along n_k) x 1 slab, 128-byte swizzle.
bool encode_bf16_slabs(CUtensorMap* m, const void* base, int64_t u, int64_t nk, int64_t v) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)v, (cuuint64_t)nk, (cuuint64_t)u};
  const cuuint64_t strides[2] = {(cuuint64_t)v * 2, (cuuint64_t)nk * (cuuint64_t)v * 2};
  const cuuint32_t box[3] = {64, (cuuint32_t)kTcK, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Row-major rows x cols FP32 matrix read in boxes of box_rows x 32 (128-byte
// rows), 128-byte swizzle, zero fill outside.
bool encode_f32_rows(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int64_t stride, int box_rows) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)stride * 4};
  const cuuint32_t box[2] = {(cuuint32_t)kTcKf, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int64_t round_up(int64_t x, int64_t q) { return (x + q - 1) / q * q; }

int64_t tc_tiles(const Shape& s) { return s.v == 1 ? (s.u + kTcRows - 1) / kTcRows : s.u * ((s.v + kTcRows - 1) / kTcRows); }

struct TcLayout {
  int Rp = 0, stages = 0, ncols = 0;
  int64_t nkp = 0;
  uint32_t stage_bytes = 0;
  size_t smem = 0, ws = 0;
};

// FP32 storage: stage = A (high part) tile + A_lo tile + X_hi / X_lo tile.
TcLayout tc_layout_f32(const Shape& s, int64_t R) {
  TcLayout L;
  L.Rp = (int)round_up(R, 16);
  L.ncols = 32;
  while (L.ncols < 2 * L.Rp) L.ncols *= 2;
  L.nkp = round_up(s.nk, kTcKf);
  L.stage_bytes = (uint32_t)(2 * kTileAf + 2 * L.Rp * 128);
  // rows (TMA tiles of A): about 110 KB of stages, two CTAs per SM (measured
  // on 65536x16384, R = 8: 5.8 TB/s; one CTA with 5 stages 3.8, three with 2
  // stages 4.2).  Slabs (A in registers one stage ahead): kStagesMN stages.
  L.stages = s.v > 1 ? kStagesMN
                     : (int)std::max<int64_t>(2, std::min<int64_t>(6, (int64_t)(110 * 1024) / L.stage_bytes));
  L.smem = 1024 + (size_t)L.stages * L.stage_bytes + (3 * (size_t)L.stages + 2) * 8;
  L.ws = align_up((size_t)2 * L.Rp * L.nkp * 4, 256);
  return L;
}

TcLayout tc_layout(const Shape& s, int64_t R) {
  TcLayout L;
  L.Rp = (int)round_up(R, 16);
  L.ncols = 32;
  while (L.ncols < 3 * L.Rp) L.ncols *= 2;  // the three pieces' accumulators
  L.nkp = round_up(s.nk, kTcK);
  L.stage_bytes = (uint32_t)(kTileA + 3 * L.Rp * 128);
  L.stages = (int)std::max<int64_t>(2, std::min<int64_t>(6, (int64_t)(96 * 1024) / L.stage_bytes));
  L.smem = 1024 + (size_t)L.stages * L.stage_bytes + (2 * (size_t)L.stages + 2) * 8;
  // at most 512 / ncols CTAs may hold tensor memory on an SM at once: ask for
  // enough shared memory that no more become resident (a further CTA's
  // allocation would wait for one of them to finish)
  const size_t per_sm = 228 * 1024;
  const size_t most = (size_t)(512 / L.ncols);
  L.smem = std::max(L.smem, per_sm / (most + 1) + 1024);
  L.ws = align_up((size_t)3 * L.Rp * L.nkp * 2, 256);
  return L;
}

}  // namespace

bool tmc_tc_supported(const Shape& s, int64_t R, tvc_dtype dt, const void* A, bool a16) {
  if (dt == TVC_F32) {
    // FP32 (tf32 parts): rows of the last mode (TMA tiles, n_k % 4 == 0), or
    // slabs at least 32 wide with v % 4 == 0 (16-byte loads by the converter
    // warps) for R > 8 (at R = 8 the CUDA-core column kernel is faster there);
    // A 16-byte aligned
    if (R < 8 || R > 64) return false;
    if (s.v == 1 ? (s.mode < 1 || s.nk % 4 != 0) : (s.v < 32 || s.v % 4 != 0 || R == 8)) return false;
    if (s.nk >= ((int64_t)1 << 31) || s.u >= ((int64_t)1 << 31) || s.v >= ((int64_t)1 << 31)) return false;
    if (!(A == nullptr ? a16 : aligned(A, 16))) return false;
    return tc_tiles(s) >= device_sms();
  }
  if (dt != TVC_BF16 || R < 8 || R > 64) return false;
  if (s.nk >= ((int64_t)1 << 31) || s.u >= ((int64_t)1 << 31) || s.v >= ((int64_t)1 << 31)) return false;
  if (s.v == 1) {
    // rows of the last mode: the contracted index is contiguous (K-major)
    if (s.mode < 1 || s.nk % 8 != 0) return false;
  } else {
    // slabs n_k x v with v contiguous (MN-major): 16-byte rows along v
    if (s.v % 8 != 0 || s.v < 64) return false;
  }
  if (!(A == nullptr ? a16 : aligned(A, 16))) return false;
  return tc_tiles(s) >= device_sms();  // enough 128-output tiles to fill the GPU
}

size_t tmc_tc_ws_bytes(const Shape& s, int64_t R, tvc_dtype dt) {
  return dt == TVC_F32 ? tc_layout_f32(s, R).ws : tc_layout(s, R).ws;
}

tvc_status tmc_tc_launch_f32(const void* A, const Shape& s, const float* X, int64_t R, float* Y, double alpha,
                             double beta, void* ws, size_t ws_bytes, cudaStream_t st) {
  const TcLayout L = tc_layout_f32(s, R);
  if (!ws || ws_bytes < L.ws || !aligned(ws, 256)) return TVC_ERR_WORKSPACE;
  float* pieces = static_cast<float*>(ws);
  const bool mn = s.v > 1;
  CUtensorMap mapA, mapX;
  if (!encode_f32_rows(&mapX, pieces, 2 * (int64_t)L.Rp, L.nkp, L.nkp, 2 * L.Rp)) return TVC_ERR_UNSUPPORTED;
  if (mn)
    mapA = mapX;  // unused: the converter warps read the slabs
  else if (!encode_f32_rows(&mapA, A, s.u, s.nk, s.nk, kTcRows))
    return TVC_ERR_UNSUPPORTED;
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    cudaFuncSetAttribute(reinterpret_cast<const void*>(tmc_tc_f32_kernel<false>),
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    cudaFuncSetAttribute(reinterpret_cast<const void*>(tmc_tc_f32_kernel<true>),
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  });
  const int64_t n = (int64_t)L.Rp * L.nkp;
  const int sblocks = (int)std::min<int64_t>((n + 255) / 256, 4LL * device_sms());
  tmc_tc_split_x_f32_kernel<<<sblocks, 256, 0, st>>>(X, pieces, R, s.nk, L.Rp, L.nkp);
  TcArgs a;
  a.Y = Y;
  a.scales = nullptr;
  a.u = s.u;
  a.R = R;
  a.upi0 = 1;
  a.v = s.v;
  a.vt = (s.v + kTcRows - 1) / kTcRows;
  a.A = static_cast<const float*>(A);
  a.nk = s.nk;
  a.Rp = L.Rp;
  a.nkb = (int)(L.nkp / kTcKf);
  a.stages = L.stages;
  a.ncols = L.ncols;
  a.stage_bytes = L.stage_bytes;
  a.alpha = (float)alpha;
  a.beta = (float)beta;
  const int64_t tiles = tc_tiles(s);
  if (tiles > 0x7FFFFFFF) return TVC_ERR_UNSUPPORTED;
  if (mn)
    tmc_tc_f32_kernel<true><<<(unsigned)tiles, kTcThreadsF, L.smem, st>>>(mapA, mapX, a);
  else
    tmc_tc_f32_kernel<false><<<(unsigned)tiles, kTcThreadsF, L.smem, st>>>(mapA, mapX, a);
  count_launches(2);
  return cuda_status(cudaGetLastError());
}

tvc_status tmc_tc_launch(const void* A, const Shape& s, const float* X, int64_t R, float* Y, const float* scales,
                         double alpha, double beta, void* ws, size_t ws_bytes, cudaStream_t st) {
  const TcLayout L = tc_layout(s, R);
  if (!ws || ws_bytes < L.ws || !aligned(ws, 256)) return TVC_ERR_WORKSPACE;
  uint16_t* pieces = static_cast<uint16_t*>(ws);
  const bool mn = s.v > 1;
  CUtensorMap mapA, mapX;
  const bool okA = mn ? encode_bf16_slabs(&mapA, A, s.u, s.nk, s.v) : encode_bf16_rows(&mapA, A, s.u, s.nk, s.nk, kTcRows);
  if (!okA || !encode_bf16_rows(&mapX, pieces, 3 * (int64_t)L.Rp, L.nkp, L.nkp, L.Rp)) return TVC_ERR_UNSUPPORTED;
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    cudaFuncSetAttribute(reinterpret_cast<const void*>(tmc_tc_kernel<false>),
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(reinterpret_cast<const void*>(tmc_tc_kernel<true>),
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  // mode 0: the slab scale belongs to the contracted index j; fold it into X
  const bool fold = s.mode == 0 && scales != nullptr;
  const int64_t n = (int64_t)L.Rp * L.nkp;
  const int sblocks = (int)std::min<int64_t>((n + 255) / 256, 4LL * device_sms());
  tmc_tc_split_x_kernel<<<sblocks, 256, 0, st>>>(X, pieces, R, s.nk, L.Rp, L.nkp, fold ? scales : nullptr);
  TcArgs a;
  a.Y = Y;
  a.scales = fold ? nullptr : scales;
  a.u = s.u;
  a.R = R;
  a.upi0 = s.upi0 > 0 ? s.upi0 : 1;
  a.v = s.v;
  a.vt = (s.v + kTcRows - 1) / kTcRows;
  a.Rp = L.Rp;
  a.nkb = (int)(L.nkp / kTcK);
  a.stages = L.stages;
  a.ncols = L.ncols;
  a.stage_bytes = L.stage_bytes;
  a.alpha = (float)alpha;
  a.beta = (float)beta;
  const int64_t tiles = tc_tiles(s);
  if (tiles > 0x7FFFFFFF) return TVC_ERR_UNSUPPORTED;
  if (mn)
    tmc_tc_kernel<true><<<(unsigned)tiles, kTcThreads, L.smem, st>>>(mapA, mapX, a);
  else
    tmc_tc_kernel<false><<<(unsigned)tiles, kTcThreads, L.smem, st>>>(mapA, mapX, a);
  count_launches(2);
  return cuda_status(cudaGetLastError());
}

// Sticky error word of the tensor-core kernel's bounded waits.
tvc_status tmc_tc_device_error(int* code_out, int clear) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tmc_tc_error, sizeof(int)) != cudaSuccess) return TVC_ERR_CUDA;
  if (clear && v) {
    const int z = 0;
    if (cudaMemcpyToSymbol(g_tmc_tc_error, &z, sizeof(int)) != cudaSuccess) return TVC_ERR_CUDA;
  }
  if (code_out) *code_out = v;
  return TVC_OK;
}

}  // namespace tvcg
