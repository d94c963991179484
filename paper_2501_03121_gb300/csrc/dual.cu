// One pass over a matrix M (R x C, row-major, FP32 / BF16 / F16 / E4M3
// storage) for the two products a Jacobi HOPM sweep needs from A:
//     T[r] = sum_c M[r,c] x[c]          (A x_{d-1} x_{d-1})
//     z[c] = sum_r w[r] M[r,c]          (A^T (x_0 (x) ... (x) x_{d-2}))
// Each 16-byte piece of M is loaded once and used for both.
//
// Mapping: the C columns are cut into chunks of CH = 32*VEC (one 16-byte
// load per lane); WG warps of a block share a row, each taking K chunks,
// and the 8/WG row groups of the block take interleaved rows of the block's
// contiguous row range.  A lane keeps its x entries and its z accumulators
// (FP32, folded every 64 rows into a compensated pair) in registers for the
// whole block, so the z products need no shared memory.  A row's dot product
// is reduced within the warp; with WG > 1 the WG partials go to Tp and a
// second kernel sums them in warp order.  The block's z partial is combined
// in row-group order in shared memory and written per block; a third kernel
// sums the blocks in order.  Every result is deterministic.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace tvcg {

namespace {

constexpr int kDualThreads = 256;
constexpr int kDualWarps = kDualThreads / kWarp;
constexpr int kDualFold = 64;  // rows between folds of the z accumulators

__device__ __forceinline__ float dual_warp_sum(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
  return v;
}

__device__ __forceinline__ bool dual_skip(const int* done) {
  return done != nullptr && *reinterpret_cast<const volatile int*>(done) != 0;
}

struct DualArgs {
  const void* M;
  int64_t R, C;
  int WG;                 // warps per row (1, 2, 4, 8)
  int64_t rows_per_block;
  const float* x;         // C
  const float* w;         // R (slab scales folded in by the caller)
  const float* scales;    // nullable: T[r] *= scales[r / upi0]
  int64_t upi0;
  float* T;               // R (written directly when WG == 1)
  float* Tp;              // WG x R partials when WG > 1
  float* P;               // gridDim.x x C block partials of z
  const int* done;
};

template <tvc_dtype DT, int VEC, int K, int UR>
__global__ void __launch_bounds__(kDualThreads) dual_kernel(const DualArgs a) {
  if (dual_skip(a.done)) return;
  using E = Elem<DT>;
  using T = typename E::T;
  constexpr int CH = kWarp * VEC;
  extern __shared__ float zsm[];  // C floats
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & (kWarp - 1);
  const int WG = a.WG, RG = kDualWarps / WG;
  const int g = warp / WG, cw = warp - (warp / WG) * WG;
  const int64_t r0 = (int64_t)blockIdx.x * a.rows_per_block;
  const int64_t r1 = min(a.R, r0 + a.rows_per_block);
  const T* M = static_cast<const T*>(a.M);
  float xr[K][VEC], za[K][VEC], zS[K][VEC], zC[K][VEC];
#pragma unroll
  for (int k = 0; k < K; k++) {
    const int64_t c = (int64_t)(cw + WG * k) * CH + lane * VEC;
#pragma unroll
    for (int e = 0; e < VEC; e++) {
      xr[k][e] = __ldg(a.x + c + e);
      za[k][e] = zS[k][e] = zC[k][e] = 0.0f;
    }
  }
  auto fold = [&]() {
#pragma unroll
    for (int k = 0; k < K; k++)
#pragma unroll
      for (int e = 0; e < VEC; e++) {
        float t, err;
        two_sum(zS[k][e], za[k][e], t, err);
        zS[k][e] = t;
        zC[k][e] = __fadd_rn(zC[k][e], err);
        za[k][e] = 0.0f;
      }
  };
  int cnt = 0;
  for (int64_t r = r0 + g; r < r1; r += UR * RG) {
    // UR rows of the group per step: their loads are in flight together
    int64_t rr[UR];
#pragma unroll
    for (int u = 0; u < UR; u++) rr[u] = r + (int64_t)u * RG;
    uint4 raw[UR][K];
    float wr[UR];
#pragma unroll
    for (int u = 0; u < UR; u++) {
      const bool ok = rr[u] < r1;
      wr[u] = ok ? __ldg(a.w + rr[u]) : 0.0f;
#pragma unroll
      for (int k = 0; k < K; k++) {
        const int64_t c = (int64_t)(cw + WG * k) * CH + lane * VEC;
        raw[u][k] = ok ? ld_stream<16>(M + rr[u] * a.C + c).v : make_uint4(0, 0, 0, 0);
      }
    }
#pragma unroll
    for (int u = 0; u < UR; u++) {
      float t = 0.0f;
#pragma unroll
      for (int k = 0; k < K; k++) {
        float v[VEC];
        E::decode16(raw[u][k], v);
#pragma unroll
        for (int e = 0; e < VEC; e++) {
          t = __fmaf_rn(v[e], xr[k][e], t);
          za[k][e] = __fmaf_rn(v[e], wr[u], za[k][e]);
        }
      }
      t = dual_warp_sum(t);
      if (lane == 0 && rr[u] < r1) {
        if (WG == 1) {
          const float sc = a.scales ? __ldg(a.scales + rr[u] / a.upi0) : 1.0f;
          a.T[rr[u]] = __fmul_rn(t, sc);
        } else {
          a.Tp[(int64_t)cw * a.R + rr[u]] = t;
        }
      }
    }
    if (++cnt == kDualFold / UR) {
      fold();
      cnt = 0;
    }
  }
  fold();
  // z partial of the block: row groups added in order (deterministic)
  for (int64_t c = threadIdx.x; c < a.C; c += kDualThreads) zsm[c] = 0.0f;
  __syncthreads();
  for (int gg = 0; gg < RG; gg++) {
    if (g == gg) {
#pragma unroll
      for (int k = 0; k < K; k++) {
        const int64_t c = (int64_t)(cw + WG * k) * CH + lane * VEC;
#pragma unroll
        for (int e = 0; e < VEC; e++) zsm[c + e] = __fadd_rn(zsm[c + e], __fadd_rn(zS[k][e], zC[k][e]));
      }
    }
    __syncthreads();
  }
  float* P = a.P + (int64_t)blockIdx.x * a.C;
  for (int64_t c = threadIdx.x; c < a.C; c += kDualThreads) P[c] = zsm[c];
}

// T[r] = (sum over the WG partials, in warp order) * scale of r's slab.
__global__ void dual_rows_kernel(const float* __restrict__ Tp, float* __restrict__ T, int64_t R, int WG,
                                 const float* scales, int64_t upi0, const int* done) {
  if (dual_skip(done)) return;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int q = 0; q < WG; q++) s = __fadd_rn(s, Tp[(int64_t)q * R + r]);
    T[r] = scales ? __fmul_rn(s, __ldg(scales + r / upi0)) : s;
  }
}

// z[c] = sum over blocks b (ascending, compensated) of P[b][c].
__global__ void dual_cols_kernel(const float* __restrict__ P, float* __restrict__ z, int64_t C, int nblk,
                                 const int* done) {
  if (dual_skip(done)) return;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
    KahanF32 s;
    for (int b = 0; b < nblk; b++) s.add(P[(int64_t)b * C + c]);
    z[c] = s.value();
  }
}

// Largest warps per row and rows in flight per warp of the single-pass
// kernel, as measured on 2048^3 and 256^4: at most 4 warps per row; 4 rows in
// flight, 2 when a lane holds 16 FP32 columns (155 registers with 4).
int dual_wg_max() { return 4; }

int dual_ur(int K, int vec) { return (vec == 4 && K * vec >= 16) ? 2 : 4; }

struct DualPlan {
  bool ok = false;
  int vec = 0, K = 0, WG = 0, grid = 0;
  int64_t rows_per_block = 0;
  size_t off_Tp = 0, off_P = 0, total = 0;
};

DualPlan dual_plan(int64_t R, int64_t C, tvc_dtype dt, const void* M) {
  DualPlan p;
  if (!(dt == TVC_F32 || dt == TVC_BF16 || dt == TVC_F16 || dt == TVC_E4M3)) return p;
  const int es = (int)elem_size(dt);
  p.vec = 16 / es;
  const int64_t CH = (int64_t)kWarp * p.vec;
  if (C % CH != 0 || !aligned(M, 16) || R < 1) return p;
  const int64_t nch = C / CH;
  int WG = dual_wg_max();
  while (WG > 1 && nch % WG != 0) WG >>= 1;
  const int64_t K = nch / WG;
  // at most 16 columns per lane (x, z and its compensation in registers)
  if (!(K == 1 || K == 2 || K == 4) || K * p.vec > 16) return p;
  p.K = (int)K;
  p.WG = WG;
  const int sms = device_sms();
  const int per_sm = (K * p.vec > 8) ? 2 : 4;
  p.grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * per_sm, (R + 63) / 64));
  p.rows_per_block = (R + p.grid - 1) / p.grid;
  size_t off = 0;
  p.off_Tp = off;
  if (WG > 1) off += align_up((size_t)WG * R * 4, 256);
  p.off_P = off;
  off += align_up((size_t)p.grid * C * 4, 256);
  p.total = off;
  p.ok = (size_t)C * 4 <= 96 * 1024;  // the block's z partial in shared memory
  return p;
}

template <tvc_dtype DT, int VEC>
void dual_go(const DualPlan& p, const DualArgs& a, size_t smem, cudaStream_t st) {
  auto go = [&](auto kern) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<p.grid, kDualThreads, smem, st>>>(a);
  };
  // K * VEC <= 16 (the planner's limit)
  const bool u4 = dual_ur(p.K, VEC) == 4;
  if (p.K == 1) {
    if (u4) go(dual_kernel<DT, VEC, 1, 4>);
    else go(dual_kernel<DT, VEC, 1, 2>);
  } else if constexpr (VEC <= 8) {
    if (p.K == 2) {
      if (u4) go(dual_kernel<DT, VEC, 2, 4>);
      else go(dual_kernel<DT, VEC, 2, 2>);
    } else if constexpr (VEC <= 4) {
      if (u4) go(dual_kernel<DT, VEC, 4, 4>);
      else go(dual_kernel<DT, VEC, 4, 2>);
    }
  }
}

}  // namespace

size_t dual_ws_bytes(int64_t R, int64_t C, tvc_dtype dt, const void* M) {
  size_t need = 0;
  for (uintptr_t al = 16; al <= 256; al *= 2) {  // any 16-byte aligned M
    const DualPlan p = dual_plan(R, C, dt, reinterpret_cast<const void*>(al));
    if (p.ok) need = std::max(need, p.total);
  }
  (void)M;
  return need;
}

bool dual_supported(int64_t R, int64_t C, tvc_dtype dt, const void* M) { return dual_plan(R, C, dt, M).ok; }

tvc_status dual_launch(const void* M, int64_t R, int64_t C, tvc_dtype dt, const float* x, const float* w,
                       const float* scales, int64_t upi0, float* T, float* z, void* ws, size_t ws_bytes,
                       cudaStream_t st, const int* done) {
  const DualPlan p = dual_plan(R, C, dt, M);
  if (!p.ok) return TVC_ERR_UNSUPPORTED;
  if (ws == nullptr || ws_bytes < p.total) return TVC_ERR_WORKSPACE;
  char* wsb = static_cast<char*>(ws);
  DualArgs a;
  a.M = M;
  a.R = R;
  a.C = C;
  a.WG = p.WG;
  a.rows_per_block = p.rows_per_block;
  a.x = x;
  a.w = w;
  a.scales = scales;
  a.upi0 = upi0 > 0 ? upi0 : 1;
  a.T = T;
  a.Tp = reinterpret_cast<float*>(wsb + p.off_Tp);
  a.P = reinterpret_cast<float*>(wsb + p.off_P);
  a.done = done;
  const size_t smem = (size_t)C * 4;
  switch (dt) {
    case TVC_F32: dual_go<TVC_F32, 4>(p, a, smem, st); break;
    case TVC_BF16: dual_go<TVC_BF16, 8>(p, a, smem, st); break;
    case TVC_F16: dual_go<TVC_F16, 8>(p, a, smem, st); break;
    default: dual_go<TVC_E4M3, 16>(p, a, smem, st); break;
  }
  int launches = 2;
  if (p.WG > 1) {
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((R + 255) / 256, 8192));
    dual_rows_kernel<<<blocks, 256, 0, st>>>(a.Tp, T, R, p.WG, scales, a.upi0, done);
    launches++;
  }
  const int cblocks = (int)std::max<int64_t>(1, std::min<int64_t>((C + 255) / 256, 1024));
  dual_cols_kernel<<<cblocks, 256, 0, st>>>(a.P, z, C, p.grid, done);
  count_launches(launches);
  return cuda_status(cudaGetLastError());
}

}  // namespace tvcg
