// Mode-k tensor-matrix contraction (the TMC of Section 1, the building
// block of the higher-order orthogonal iteration for the Tucker
// decomposition and of CP alternating least squares):
//     Y[i][r][l] = alpha * sum_{j < n_k} A[i][j][l] X[r][j] + beta * Y[i][r][l]
// for an R x n_k matrix X, with A read as u x n_k x v (Section 3) and Y of
// the shape of A with n_k replaced by R (row-major).
//
// Like the TVC it streams A once in its own order whatever k is; RP rows of
// X (4, 8 or 16) are applied per pass over A (blockIdx.z), and the rows of X
// are staged in shared memory (16 KB chunks of the n_k range, one block
// barrier per chunk), read by broadcast or shared by a warp's rows.  The
// kernels:
//   * tmc_cols_async_kernel (FP32, v > 1): a thread owns 16/RP output
//     columns (i, l..) and keeps the next rows of that piece in flight with
//     cp.async into its own shared-memory slots;
//   * tmc_rows_group_kernel (v == 1, FP32 and narrow storage): a few lanes
//     per row read 16-byte pieces along it with a cp.async pipeline, and
//     the RP partial sums are reduced over the lanes by a butterfly;
//   * tmc_f64_kernel (FP64, single-double): float-float products on the
//     FP32 pipe, FP64 totals;
//   * tmc_kernel: every other case, one output column per thread, 16 (8)
//     rows in flight.
// Few outputs split n_k over blockIdx.y; tmc_reduce_kernel adds the partial
// sums in a fixed order (deterministic).  FP32 accumulation is two-level
// (64 products, then the running sum).
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "tma.cuh"

namespace tvcg {
namespace {

constexpr int kTmcThreads = 256;
constexpr int kXsBytes = 16 * 1024;  // shared memory for the staged rows of X

template <tvc_dtype DT>
using TmcW = std::conditional_t<kF64Acc<DT>, double, float>;  // vectors and accumulators

template <tvc_dtype DT>
struct TmcArgs {
  const typename Elem<DT>::T* A;
  const TmcW<DT>* X;    // R x nk
  const float* scales;  // narrow types, nullable
  TmcW<DT>* Y;          // u x R x v
  TmcW<DT>* partial;    // splits x (u R v) when splits > 1
  int64_t u, nk, v, uv, R, upi0, chunk, uRv;
  int mode0, splits, jc;  // jc: entries j of X staged at a time (a multiple of 16)
  double alpha, beta;
};

// U entries of one output column: rows j .. j+U-1 at stride v (streaming
// loads), or (VJ) the contiguous run p[0..U-1] of a row (v == 1, U-element
// aligned) with L1-cached 16-byte loads, so that the 32-byte sector a
// thread's row piece shares with nothing else stays in L1 between its loads.
template <tvc_dtype DT, bool VJ, int U>
__device__ __forceinline__ void loadU(const typename Elem<DT>::T* p, int64_t v, typename Elem<DT>::C (&r)[U]) {
  using E = Elem<DT>;
  if constexpr (VJ) {
    constexpr int P = 16 / E::kSize;  // elements per 16-byte piece
    static_assert(U % P == 0, "U must be a multiple of the 16-byte piece");
#pragma unroll
    for (int h = 0; h < U / P; h++) {
      typename E::C t[P];
      E::template load<P, true>(p + P * h, t);
#pragma unroll
      for (int e = 0; e < P; e++) r[P * h + e] = t[e];
    }
  } else {
#pragma unroll
    for (int q = 0; q < U; q++) {
      typename E::C t[1];
      E::template load<1>(p + q * v, t);
      r[q] = t[0];
    }
  }
}

// Two FP32 fused multiply-adds in one instruction (the paired FP32 pipe of
// sm_100 and later): each lane is an IEEE fma with round-to-nearest, so the
// results equal two separate fmaf calls.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long ua, ub, uc, ud;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ua) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(ub) : "f"(b.x), "f"(b.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(uc) : "f"(c.x), "f"(c.y));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(ud) : "l"(ua), "l"(ub), "l"(uc));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(ud));
  return d;
}

// acc[r] += a * Xs[j][r] for r < RP, Xs read in 16-byte pieces; up to 8
// rows of X the products go in pairs of rows (fma2: measured 1.4x for BF16
// columns at R = 8, but 0.9x at R = 16, which keeps single multiply-adds).
template <int RP, class W, class C>
__device__ __forceinline__ void mac_row(W (&acc)[RP], C a, const W* xs) {
  if constexpr (sizeof(W) == 4 && RP > 8) {
#pragma unroll
    for (int r = 0; r < RP; r += 4) {
      const float4 xv = *reinterpret_cast<const float4*>(xs + r);
      acc[r] = __fmaf_rn(a, xv.x, acc[r]);
      acc[r + 1] = __fmaf_rn(a, xv.y, acc[r + 1]);
      acc[r + 2] = __fmaf_rn(a, xv.z, acc[r + 2]);
      acc[r + 3] = __fmaf_rn(a, xv.w, acc[r + 3]);
    }
  } else if constexpr (sizeof(W) == 4) {
    const float2 aa = make_float2(a, a);
#pragma unroll
    for (int r = 0; r < RP; r += 4) {
      const float4 xv = *reinterpret_cast<const float4*>(xs + r);
      const float2 p0 = fma2(aa, make_float2(xv.x, xv.y), make_float2(acc[r], acc[r + 1]));
      const float2 p1 = fma2(aa, make_float2(xv.z, xv.w), make_float2(acc[r + 2], acc[r + 3]));
      acc[r] = p0.x;
      acc[r + 1] = p0.y;
      acc[r + 2] = p1.x;
      acc[r + 3] = p1.y;
    }
  } else {
#pragma unroll
    for (int r = 0; r < RP; r += 2) {
      const double2 xv = *reinterpret_cast<const double2*>(xs + r);
      acc[r] = fma((double)a, xv.x, acc[r]);
      acc[r + 1] = fma((double)a, xv.y, acc[r + 1]);
    }
  }
}

// Rows of A in flight per thread: 16 when the accumulators leave room.
template <tvc_dtype DT, int RP>
inline constexpr int kTmcU = (RP * sizeof(TmcW<DT>) <= 32) ? 16 : 8;

template <tvc_dtype DT, int RP, bool VJ>
__global__ void __launch_bounds__(kTmcThreads) tmc_kernel(const TmcArgs<DT> a) {
  using E = Elem<DT>;
  using T = typename E::T;
  using C = typename E::C;
  using W = TmcW<DT>;
  constexpr bool kF32 = sizeof(W) == 4;
  extern __shared__ __align__(16) unsigned char xs_raw[];
  W* Xs = reinterpret_cast<W*>(xs_raw);  // [jc][RP]
  const int64_t o = (int64_t)blockIdx.x * kTmcThreads + threadIdx.x;  // output column (i, l)
  const bool act = o < a.uv;
  const int64_t i = act ? o / a.v : 0;
  const int64_t l = act ? o - i * a.v : 0;
  const int64_t r0 = (int64_t)blockIdx.z * RP;
  const int64_t j0 = (int64_t)blockIdx.y * a.chunk;
  const int64_t j1 = min(a.nk, j0 + a.chunk);
  const T* p = a.A + (i * a.nk + j0) * a.v + l;
  W acc[RP], sum[RP];
#pragma unroll
  for (int r = 0; r < RP; r++) {
    acc[r] = 0;
    sum[r] = 0;
  }
  const bool fold_scale = kNarrow<DT> && a.mode0 && a.scales;
  int blk = 0;
  for (int64_t jc = j0; jc < j1; jc += a.jc) {
    const int jn = (int)min((int64_t)a.jc, j1 - jc);
    __syncthreads();  // the previous chunk is consumed
    for (int t = threadIdx.x; t < jn * RP; t += kTmcThreads) {
      const int jl = t / RP, r = t - (t / RP) * RP;
      W xv = 0;
      if (r0 + r < a.R) {
        xv = a.X[(r0 + r) * a.nk + jc + jl];
        if (fold_scale) xv *= (W)__ldg(a.scales + jc + jl);  // k = 0: row j lies in slab j
      }
      Xs[t] = xv;
    }
    __syncthreads();
    if (act) {
      constexpr int P16 = 16 / Elem<DT>::kSize;
      constexpr int U = (VJ && kTmcU<DT, RP> < P16) ? P16 : kTmcU<DT, RP>;
      int jl = 0;
      for (; jl + U <= jn; jl += U) {
        C vu[U];
        loadU<DT, VJ, U>(p, a.v, vu);
#pragma unroll
        for (int q = 0; q < U; q++) mac_row<RP>(acc, vu[q], Xs + (jl + q) * RP);
        p += U * a.v;
        if constexpr (kF32) {
          if (++blk == 64 / U) {  // 64 products per partial sum
#pragma unroll
            for (int r = 0; r < RP; r++) {
              sum[r] += acc[r];
              acc[r] = 0;
            }
            blk = 0;
          }
        }
      }
      for (; jl < jn; jl++, p += a.v) {
        C v1[1];
        E::template load<1>(p, v1);
        mac_row<RP>(acc, v1[0], Xs + jl * RP);
      }
    }
  }
  if (!act) return;
  W sc = 1;
  if constexpr (kNarrow<DT>) {
    if (!a.mode0 && a.scales) sc = (W)__ldg(a.scales + i / a.upi0);
  }
#pragma unroll
  for (int r = 0; r < RP; r++) {
    if (r0 + r < a.R) {
      const W val = (sum[r] + acc[r]) * sc;
      const int64_t y = (i * a.R + r0 + r) * a.v + l;
      if (a.splits > 1) {
        a.partial[blockIdx.y * a.uRv + y] = val;
      } else {
        W out = (W)a.alpha * val;
        if (a.beta != 0.0) out += (W)a.beta * a.Y[y];
        a.Y[y] = out;
      }
    }
  }
}

// FP64 and single-double storage: the products on the FP32 pipe in
// float-float arithmetic, as in the TVC's FP64 kernels (one DFMA per
// product would leave an FP64 TMC at a fraction of the bandwidth: the
// FP64 pipe runs about two multiply-adds per SM per clock).  Each element
// a is split once into ah + al (exact in the window 2^-64 <= |a| < 2^64);
// each row r of X was split into xh + xl when staged; the product's error
// terms go into a compensated pair (s_r, c_r), folded into an FP64 total
// every 64 products.  Nonzero elements or entries of X outside their
// windows (NaN pieces for X) flag the thread, which then recomputes its
// outputs with FP64 multiply-adds: exact-window results are FP64-accurate,
// the rest are the plain FP64 dot products.
template <int RP>
__device__ __forceinline__ void df_row(float (&s)[RP], float (&c)[RP], float ah, float al, const float2* xs) {
#pragma unroll
  for (int r = 0; r < RP; r += 2) {
    const float4 x2 = *reinterpret_cast<const float4*>(xs + r);  // (xh, xl) of rows r, r + 1
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const float xh = h ? x2.z : x2.x, xl = h ? x2.w : x2.y;
      const float pr = __fmul_rn(ah, xh);
      float e = __fmaf_rn(ah, xh, -pr);
      e = __fmaf_rn(ah, xl, e);
      e = __fmaf_rn(al, xh, e);
      float t, err;
      two_sum(s[r + h], pr, t, err);
      s[r + h] = t;
      c[r + h] = __fadd_rn(c[r + h], __fadd_rn(err, e));
    }
  }
}

// Pieces of one element; zeros are exact (0 + 0), other elements outside
// the window set `bad`.
__device__ __forceinline__ void split_elem(double v, float& ah, float& al, uint32_t& bad) {
  const bool z = v == 0.0;
  bad |= (df_out_of_window(v) != 0u && !z) ? 1u : 0u;
  df_split(v, ah, al);
  ah = z ? 0.0f : ah;
  al = z ? 0.0f : al;
}
__device__ __forceinline__ void split_elem(float v, float& ah, float& al, uint32_t& bad) {
  bad |= (df_out_of_window(v) != 0u && v != 0.0f) ? 1u : 0u;
  ah = v;
  al = 0.0f;
}

template <tvc_dtype DT, int RP, bool VJ>
__global__ void __launch_bounds__(kTmcThreads) tmc_f64_kernel(const TmcArgs<DT> a) {
  using E = Elem<DT>;
  using T = typename E::T;
  using C = typename E::C;  // double (FP64) or float (single-double)
  extern __shared__ __align__(16) unsigned char xs_raw[];
  float2* Xs = reinterpret_cast<float2*>(xs_raw);  // [jc][RP] split entries of X
  const int64_t o = (int64_t)blockIdx.x * kTmcThreads + threadIdx.x;  // output column (i, l)
  const bool act = o < a.uv;
  const int64_t i = act ? o / a.v : 0;
  const int64_t l = act ? o - i * a.v : 0;
  const int64_t r0 = (int64_t)blockIdx.z * RP;
  const int64_t j0 = (int64_t)blockIdx.y * a.chunk;
  const int64_t j1 = min(a.nk, j0 + a.chunk);
  const T* p = a.A + (i * a.nk + j0) * a.v + l;
  float s[RP], c[RP];
  double d[RP];
#pragma unroll
  for (int r = 0; r < RP; r++) {
    s[r] = 0.0f;
    c[r] = 0.0f;
    d[r] = 0.0;
  }
  uint32_t bad = 0;
  constexpr int U = 8;
  int blk = 0;
  for (int64_t jc = j0; jc < j1; jc += a.jc) {
    const int jn = (int)min((int64_t)a.jc, j1 - jc);
    __syncthreads();  // the previous chunk is consumed
    for (int t = threadIdx.x; t < jn * RP; t += kTmcThreads) {
      const int jl = t / RP, r = t - (t / RP) * RP;
      XSplit xsp{0.0f, 0.0f};
      if (r0 + r < a.R) xsp = split_x(a.X[(r0 + r) * a.nk + jc + jl]);
      Xs[t] = make_float2(xsp.xh, xsp.xl);
    }
    __syncthreads();
    if (act) {
      int jl = 0;
      for (; jl + U <= jn; jl += U) {
        C vu[U];
        loadU<DT, VJ, U>(p, a.v, vu);
#pragma unroll
        for (int q = 0; q < U; q++) {
          float ah, al;
          split_elem(vu[q], ah, al, bad);
          df_row<RP>(s, c, ah, al, Xs + (jl + q) * RP);
        }
        p += U * a.v;
        if (++blk == 64 / U) {  // 64 products per compensated pair
#pragma unroll
          for (int r = 0; r < RP; r++) {
            d[r] += (double)s[r];
            d[r] += (double)c[r];
            s[r] = 0.0f;
            c[r] = 0.0f;
          }
          blk = 0;
        }
      }
      for (; jl < jn; jl++, p += a.v) {
        C v1[1];
        E::template load<1>(p, v1);
        float ah, al;
        split_elem(v1[0], ah, al, bad);
        df_row<RP>(s, c, ah, al, Xs + jl * RP);
      }
    }
  }
  if (!act) return;
  bool redo = bad != 0;
#pragma unroll
  for (int r = 0; r < RP; r++) {
    d[r] += (double)s[r];
    d[r] += (double)c[r];
    redo = redo || !isfinite(d[r]);
  }
  if (redo) {  // rare: plain FP64 multiply-adds over this thread's range
#pragma unroll
    for (int r = 0; r < RP; r++) d[r] = 0.0;
    const T* q = a.A + (i * a.nk + j0) * a.v + l;
    for (int64_t j = j0; j < j1; j++, q += a.v) {
      C v1[1];
      E::template load<1>(q, v1);
#pragma unroll
      for (int r = 0; r < RP; r++)
        if (r0 + r < a.R) d[r] = fma((double)v1[0], a.X[(r0 + r) * a.nk + j], d[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < RP; r++) {
    if (r0 + r < a.R) {
      const int64_t y = (i * a.R + r0 + r) * a.v + l;
      if (a.splits > 1) {
        a.partial[blockIdx.y * a.uRv + y] = d[r];
      } else {
        double out = a.alpha * d[r];
        if (a.beta != 0.0) out += a.beta * a.Y[y];
        a.Y[y] = out;
      }
    }
  }
}

// FP32 storage, v % VEC == 0: each thread owns VEC = 16 / RP consecutive
// output columns (i, l..l+VEC-1) and keeps the next D rows of that piece
// (4 * VEC bytes) in flight with cp.async into its own shared-memory slots,
// consuming row j while row j + D is fetched (it waits only for its own
// copies).  VEC x RP accumulators (two levels), X staged as in tmc_kernel.
// A column piece of 4, 8 or 16 bytes.
template <int BYTES>
__device__ __forceinline__ void cp_async_piece(void* smem, const void* gmem) {
  if constexpr (BYTES == 16)
    cp_async16(smem, gmem);
  else if constexpr (BYTES == 8)
    cp_async8(smem, gmem);
  else
    cp_async4(smem, gmem);
}

template <int RP>
struct TmcAsync {
  static constexpr int VEC = 16 / RP;               // 4, 2, 1 floats per piece
  static constexpr int D = VEC == 4 ? 8 : 16;       // rows in flight per thread
};

template <int RP>
__global__ void __launch_bounds__(kTmcThreads) tmc_cols_async_kernel(const TmcArgs<TVC_F32> a) {
  using Q = TmcAsync<RP>;
  constexpr int VEC = Q::VEC, D = Q::D;
  __shared__ __align__(16) float stage[D][kTmcThreads * VEC];
  extern __shared__ __align__(16) unsigned char xs_raw[];
  float* Xs = reinterpret_cast<float*>(xs_raw);  // [jc][RP]
  const int t = threadIdx.x;
  const int64_t o = ((int64_t)blockIdx.x * kTmcThreads + t) * VEC;
  const bool act = o < a.uv;
  const int64_t oo = act ? o : 0;
  const int64_t i = oo / a.v;
  const int64_t l = oo - i * a.v;
  const int64_t r0 = (int64_t)blockIdx.z * RP;
  const int64_t j0 = (int64_t)blockIdx.y * a.chunk;
  const int64_t j1 = min(a.nk, j0 + a.chunk);
  const float* p = a.A + (i * a.nk + j0) * a.v + l;
  const int64_t n = act ? j1 - j0 : 0;
#pragma unroll
  for (int d = 0; d < D; d++) {
    if (d < n) cp_async_piece<VEC * 4>(&stage[d][t * VEC], p + d * a.v);
    cp_async_commit();
  }
  float acc[VEC][RP], sum[VEC][RP];
#pragma unroll
  for (int e = 0; e < VEC; e++)
#pragma unroll
    for (int r = 0; r < RP; r++) {
      acc[e][r] = 0.0f;
      sum[e][r] = 0.0f;
    }
  int slot = 0, blk = 0;
  int64_t left = n - D;           // rows still to fetch after the prologue
  const float* pf = p + D * a.v;  // next row to fetch
  for (int64_t jc = j0; jc < j1; jc += a.jc) {
    const int jn = (int)min((int64_t)a.jc, j1 - jc);
    __syncthreads();  // the previous chunk of X is consumed
    for (int q = t; q < jn * RP; q += kTmcThreads) {
      const int jl = q / RP, r = q - (q / RP) * RP;
      Xs[q] = (r0 + r < a.R) ? a.X[(r0 + r) * a.nk + jc + jl] : 0.0f;
    }
    __syncthreads();
    if (act) {
      for (int jl = 0; jl < jn; jl++) {
        cp_async_wait<D - 1>();
        float v[VEC];
        if constexpr (VEC == 4) {
          const float4 f = *reinterpret_cast<const float4*>(&stage[slot][t * 4]);
          v[0] = f.x;
          v[1] = f.y;
          v[2] = f.z;
          v[3] = f.w;
        } else if constexpr (VEC == 2) {
          const float2 f = *reinterpret_cast<const float2*>(&stage[slot][t * 2]);
          v[0] = f.x;
          v[1] = f.y;
        } else {
          v[0] = stage[slot][t];
        }
        // the slot is free again: fetch the row D ahead into it
        if (left > 0) cp_async_piece<VEC * 4>(&stage[slot][t * VEC], pf);
        cp_async_commit();
        left--;
        pf += a.v;
#pragma unroll
        for (int e = 0; e < VEC; e++) mac_row<RP>(acc[e], v[e], Xs + jl * RP);
        if (++slot == D) slot = 0;
        if (++blk == 64) {
#pragma unroll
          for (int e = 0; e < VEC; e++)
#pragma unroll
            for (int r = 0; r < RP; r++) {
              sum[e][r] += acc[e][r];
              acc[e][r] = 0.0f;
            }
          blk = 0;
        }
      }
    }
  }
  cp_async_wait<0>();
  if (!act) return;
#pragma unroll
  for (int r = 0; r < RP; r++) {
    if (r0 + r < a.R) {
#pragma unroll
      for (int e = 0; e < VEC; e++) {
        const float val = sum[e][r] + acc[e][r];
        const int64_t y = (i * a.R + r0 + r) * a.v + l + e;
        if (a.splits > 1) {
          a.partial[blockIdx.y * a.uRv + y] = val;
        } else {
          float out = (float)a.alpha * val;
          if (a.beta != 0.0) out += (float)a.beta * a.Y[y];
          a.Y[y] = out;
        }
      }
    }
  }
}

// Rows (v == 1) by lane groups: G lanes (2, 4 or 8) share one row, lane g
// reading the 16-byte pieces g, g + G, ... (P entries each), so a warp
// reads 32 / G rows as contiguous runs.  X is staged transposed, Xt[r][j],
// so a lane's P entries of row r of X are 16-byte shared-memory reads that
// the 32 / G rows of the warp share (few lanes per row keep the shared-
// memory traffic per element of A low).  Each lane keeps its next 8 pieces
// in flight with cp.async into its own shared-memory slots.  Each lane
// accumulates RP partial sums (two levels); at the end the group reduces
// them by a butterfly that halves the values a lane keeps at every level
// (RP - 1 + log2(G / RP) exchanges instead of RP log2 G), a fixed order.
// A block owns 8 * 32 / G rows for its whole n_k range (chunks of X staged
// in turn); when X fits in one chunk the block loops over further rows.
template <int G, int K>
__device__ __forceinline__ void group_reduce(float (&v)[K], int gl, int& base, bool& writer) {
  int kk = K;
  base = 0;
  writer = true;
#pragma unroll
  for (int off = G / 2; off >= 1; off >>= 1) {
    const bool hi = (gl & off) != 0;
    if (kk > 1) {
      const int half = kk / 2;
#pragma unroll
      for (int m = 0; m < K / 2; m++) {
        if (m < half) {
          const float send = hi ? v[m] : v[m + half];
          const float keep = hi ? v[m + half] : v[m];
          v[m] = __fadd_rn(keep, __shfl_xor_sync(0xFFFFFFFFu, send, off));
        }
      }
      if (hi) base += half;
      kk = half;
    } else {
      v[0] = __fadd_rn(v[0], __shfl_xor_sync(0xFFFFFFFFu, v[0], off));
      writer = writer && !hi;
    }
  }
}

constexpr int kGroupD = 8;  // 16-byte pieces in flight per lane (cp.async)

template <int RP>
inline constexpr int kGroupJC = kXsBytes / (RP * 4);  // row stride of the transposed X (entries)

template <tvc_dtype DT, int RP, int G>
__global__ void __launch_bounds__(kTmcThreads) tmc_rows_group_kernel(const TmcArgs<DT> a, int loop_rows) {
  using E = Elem<DT>;
  using T = typename E::T;
  constexpr int P = 16 / E::kSize;                    // entries per 16-byte piece
  constexpr int RPB = (kTmcThreads / 32) * (32 / G);  // rows per block
  constexpr int JT = kGroupJC<RP>;                    // a.jc <= JT
  __shared__ __align__(16) uint4 stage[kGroupD][kTmcThreads];
  extern __shared__ __align__(16) unsigned char xs_raw[];
  float* Xt = reinterpret_cast<float*>(xs_raw);  // [RP][JT]
  const int t = threadIdx.x, lane = t & 31, gl = lane & (G - 1);
  const int row_in_block = (t >> 5) * (32 / G) + (lane / G);
  const int64_t r0 = (int64_t)blockIdx.z * RP;
  const int64_t j0 = (int64_t)blockIdx.y * a.chunk;
  const int64_t j1 = min(a.nk, j0 + a.chunk);
  const int64_t pieces = (j1 - j0) / P;  // of the row in [j0, j1)
  const bool fold_scale = kNarrow<DT> && a.mode0 && a.scales;
  bool staged = false;
  for (int64_t rb = blockIdx.x; rb * RPB < a.u; rb += gridDim.x) {
    const int64_t i = rb * RPB + row_in_block;
    const bool act = i < a.u;
    const T* prow = a.A + (act ? i : 0) * a.nk + j0;
    const int64_t n = act ? (pieces > gl ? (pieces - gl + G - 1) / G : 0) : 0;  // this lane's pieces
#pragma unroll
    for (int d = 0; d < kGroupD; d++) {
      if (d < n) cp_async16(&stage[d][t], prow + (gl + (int64_t)d * G) * P);
      cp_async_commit();
    }
    float acc[RP], sum[RP];
#pragma unroll
    for (int r = 0; r < RP; r++) {
      acc[r] = 0.0f;
      sum[r] = 0.0f;
    }
    int blk = 0, slot = 0;
    int64_t k = 0;                                      // next piece of this lane
    int64_t left = n - kGroupD;                         // pieces still to fetch after the prologue
    const T* pf = prow + (gl + (int64_t)kGroupD * G) * P;  // next piece to fetch
    for (int64_t jc = j0; jc < j1; jc += a.jc) {
      const int jn = (int)min((int64_t)a.jc, j1 - jc);
      if (!(loop_rows && staged)) {
        __syncthreads();  // the previous chunk of X is consumed
        for (int q = t; q < RP * JT; q += kTmcThreads) {
          const int r = q / JT, jl = q - (q / JT) * JT;
          float xv = 0.0f;
          if (jl < jn && r0 + r < a.R) {
            xv = a.X[(r0 + r) * a.nk + jc + jl];
            if (fold_scale) xv *= __ldg(a.scales + jc + jl);  // order 1: entry j lies in slab j
          }
          Xt[q] = xv;
        }
        __syncthreads();
        staged = true;
      }
      // this lane's pieces whose entries lie in [jc, jc + jn)
      for (int jl = (int)((gl + k * G) * P - (jc - j0)); k < n && jl < jn; k++, jl += G * P) {
        cp_async_wait<kGroupD - 1>();
        float v[P];
        E::template load<P, true>(reinterpret_cast<const T*>(&stage[slot][t]), v);
        if (left > 0) cp_async16(&stage[slot][t], pf);
        cp_async_commit();
        left--;
        pf += G * P;
        if (++slot == kGroupD) slot = 0;
        const float* xj = Xt + jl;
#pragma unroll
        for (int r = 0; r < RP; r++) {
          const float* xr = xj + r * JT;
#pragma unroll
          for (int q = 0; q < P; q += 4) {
            const float4 xv = *reinterpret_cast<const float4*>(xr + q);
            acc[r] = __fmaf_rn(v[q], xv.x, acc[r]);
            acc[r] = __fmaf_rn(v[q + 1], xv.y, acc[r]);
            acc[r] = __fmaf_rn(v[q + 2], xv.z, acc[r]);
            acc[r] = __fmaf_rn(v[q + 3], xv.w, acc[r]);
          }
        }
        if (++blk == (64 + P - 1) / P) {  // about 64 products per partial sum
#pragma unroll
          for (int r = 0; r < RP; r++) {
            sum[r] += acc[r];
            acc[r] = 0.0f;
          }
          blk = 0;
        }
      }
    }
    cp_async_wait<0>();
    float tot[RP];
#pragma unroll
    for (int r = 0; r < RP; r++) tot[r] = sum[r] + acc[r];
    int base;
    bool writer;
    group_reduce<G, RP>(tot, gl, base, writer);
    constexpr int KF = (RP / G) > 1 ? RP / G : 1;
    if (act && writer) {
      float sc = 1.0f;
      if constexpr (kNarrow<DT>) {
        if (!a.mode0 && a.scales) sc = __ldg(a.scales + i / a.upi0);
      }
#pragma unroll
      for (int m = 0; m < KF; m++) {
        if (r0 + base + m < a.R) {
          const float val = tot[m] * sc;
          const int64_t y = i * a.R + r0 + base + m;
          if (a.splits > 1) {
            a.partial[blockIdx.y * a.uRv + y] = val;
          } else {
            float out = (float)a.alpha * val;
            if (a.beta != 0.0) out += (float)a.beta * a.Y[y];
            a.Y[y] = out;
          }
        }
      }
    }
    if (!loop_rows) break;
  }
}

// Y[o] = alpha * sum_s partial[s][o] + beta * Y[o], s ascending.
template <class W>
__global__ void tmc_reduce_kernel(const W* __restrict__ partial, W* __restrict__ Y, int64_t n, int splits,
                                  double alpha, double beta) {
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
    W s = 0;
    for (int k = 0; k < splits; k++) s += partial[(int64_t)k * n + o];
    W r = (W)alpha * s;
    if (beta != 0.0) r += (W)beta * Y[o];
    Y[o] = r;
  }
}

// Launch plan: rows of X per pass, passes, split of n_k.
struct TmcPlan {
  int rp = 8, passes = 1, splits = 1, jc = 8, vec = 1;
  bool async = false;       // FP32 column pieces through the cp.async pipeline
  int group = 0;            // lanes per row of the lane-group rows kernel (0: not used)
  bool loop_rows = false;   // X staged once, the block loops over row groups
  int64_t chunk = 0, blocks_x = 0;
  bool vj = false;
  bool tc = false;          // the tensor-core kernel (tmc_tc.cu)
  size_t ws = 0;
};

int tmc_rp(tvc_dtype dt, int64_t R) {
  const bool f64 = vec_size(dt) == 8;
  if (R <= 4) return 4;
  if (R <= 8 || f64) return 8;
  return 16;
}

// A == nullptr (the workspace query) plans for a 16-byte aligned A; the
// query reports the larger workspace of the aligned and unaligned plans.
TmcPlan tmc_plan(const Shape& s, int64_t R, tvc_dtype dt, const void* A, bool a16 = false) {
  TmcPlan p;
  if (tmc_tc_supported(s, R, dt, A, a16)) {
    // BF16 codes (any mode) or FP32 along the last mode with R >= 8: a
    // matrix product on the tensor cores (the CUDA-core kernels are
    // issue-bound there)
    p.tc = true;
    p.ws = tmc_tc_ws_bytes(s, R, dt);
    return p;
  }
  p.rp = tmc_rp(dt, R);
  p.passes = (int)((R + p.rp - 1) / p.rp);
  const int avec = 16 / p.rp;
  const bool f32 = dt == TVC_F32 && p.rp <= 8;
  p.async = f32 && s.v > 1 && s.v % avec == 0 && (A == nullptr ? a16 : aligned(A, 4 * avec));
  p.vec = p.async ? avec : 1;
  p.blocks_x = (s.uv / p.vec + kTmcThreads - 1) / kTmcThreads;
  // rows by lane groups: FP32-accumulated types, 16-byte pieces along rows
  const int piece = 16 / (int)elem_size(dt);
  if (vec_size(dt) == 4 && p.rp <= 8 && s.v == 1 && s.nk % piece == 0 && s.nk / piece >= 2 &&
      (A == nullptr ? a16 : aligned(A, 16))) {
    // G lanes per row: 128 contiguous bytes per row for FP32; fewer lanes
    // for the narrow types so that more rows of a warp share each read of X
    int g = elem_size(dt) == 4 ? 8 : elem_size(dt) == 2 ? 4 : 2;
    while (g > 2 && g * piece > s.nk) g /= 2;
    p.group = g;
    const int64_t rpb = (kTmcThreads / 32) * (32 / g);
    p.blocks_x = (s.u + rpb - 1) / rpb;
  }
  const int64_t want = 4LL * device_sms();  // blocks for a full GPU
  int64_t have = p.blocks_x * p.passes;
  int64_t splits = 1;
  if (have < want) splits = std::min<int64_t>((want + have - 1) / have, std::max<int64_t>(1, s.nk / 256));
  p.chunk = ((s.nk + splits - 1) / splits + 15) / 16 * 16;
  p.splits = (int)((s.nk + p.chunk - 1) / p.chunk);
  p.vj = s.v == 1 && s.nk % 16 == 0 && aligned(A, 16);
  const int jmax = kXsBytes / (p.rp * (int)vec_size(dt)) / 16 * 16;
  p.jc = (int)std::min<int64_t>(jmax, p.chunk);
  if (p.group && p.splits == 1 && p.chunk <= p.jc) {
    p.loop_rows = true;
    p.blocks_x = std::min<int64_t>(p.blocks_x, 8LL * device_sms());
  }
  p.ws = p.splits > 1 ? (size_t)p.splits * (size_t)(s.uv * R) * vec_size(dt) : 0;
  return p;
}

template <tvc_dtype DT, int RP>
void launch_rp(const TmcArgs<DT>& a, const TmcPlan& p, cudaStream_t st) {
  dim3 grid((unsigned)p.blocks_x, (unsigned)p.splits, (unsigned)p.passes);
  const size_t smem = (size_t)p.jc * RP * sizeof(TmcW<DT>);
  if constexpr (!kF64Acc<DT> && RP <= 8) {
    if (p.group) {
      const size_t gsmem = (size_t)kGroupJC<RP> * RP * sizeof(float);
      const int lr = p.loop_rows ? 1 : 0;
      switch (p.group) {
        case 2: tmc_rows_group_kernel<DT, RP, 2><<<grid, kTmcThreads, gsmem, st>>>(a, lr); break;
        case 4: tmc_rows_group_kernel<DT, RP, 4><<<grid, kTmcThreads, gsmem, st>>>(a, lr); break;
        default: tmc_rows_group_kernel<DT, RP, 8><<<grid, kTmcThreads, gsmem, st>>>(a, lr); break;
      }
      return;
    }
  }
  if constexpr (DT == TVC_F32) {
    if constexpr (RP <= 8) {
      if (p.async) {
        tmc_cols_async_kernel<RP><<<grid, kTmcThreads, smem, st>>>(a);
        return;
      }
    }
  }
  if constexpr (kF64Acc<DT>) {
    if (p.vj)
      tmc_f64_kernel<DT, RP, true><<<grid, kTmcThreads, smem, st>>>(a);
    else
      tmc_f64_kernel<DT, RP, false><<<grid, kTmcThreads, smem, st>>>(a);
    return;
  }
  if (p.vj)
    tmc_kernel<DT, RP, true><<<grid, kTmcThreads, smem, st>>>(a);
  else
    tmc_kernel<DT, RP, false><<<grid, kTmcThreads, smem, st>>>(a);
}

template <tvc_dtype DT>
tvc_status run(const void* A, const Shape& s, const void* X, int64_t R, void* Y, const float* scales, double alpha,
               double beta, void* ws, size_t ws_size, const TmcPlan& p, cudaStream_t st) {
  using W = TmcW<DT>;
  if constexpr (DT == TVC_BF16) {
    if (p.tc)
      return tmc_tc_launch(A, s, static_cast<const float*>(X), R, static_cast<float*>(Y), scales, alpha, beta, ws,
                           ws_size, st);
  }
  if constexpr (DT == TVC_F32) {
    if (p.tc)
      return tmc_tc_launch_f32(A, s, static_cast<const float*>(X), R, static_cast<float*>(Y), alpha, beta, ws,
                               ws_size, st);
  }
  TmcArgs<DT> a;
  a.A = static_cast<const typename Elem<DT>::T*>(A);
  a.X = static_cast<const W*>(X);
  a.scales = scales;
  a.Y = static_cast<W*>(Y);
  a.partial = static_cast<W*>(ws);
  a.u = s.u;
  a.nk = s.nk;
  a.v = s.v;
  a.uv = s.uv;
  a.R = R;
  a.upi0 = s.upi0;
  a.chunk = p.chunk;
  a.uRv = s.uv * R;
  a.mode0 = s.mode == 0;
  a.splits = p.splits;
  a.jc = p.jc;
  a.alpha = alpha;
  a.beta = beta;
  if (p.blocks_x > 0x7FFFFFFF || p.passes > 65535) return TVC_ERR_UNSUPPORTED;
  switch (p.rp) {
    case 4: launch_rp<DT, 4>(a, p, st); break;
    case 8: launch_rp<DT, 8>(a, p, st); break;
    default:
      if constexpr (!kF64Acc<DT>) launch_rp<DT, 16>(a, p, st);
      break;
  }
  int launches = 1;
  if (p.splits > 1) {
    const int64_t n = s.uv * R;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 8LL * device_sms());
    tmc_reduce_kernel<W><<<blocks, 256, 0, st>>>(static_cast<const W*>(ws), static_cast<W*>(Y), n, p.splits, alpha,
                                                 beta);
    launches++;
  }
  count_launches(launches);
  return cuda_status(cudaGetLastError());
}

}  // namespace
}  // namespace tvcg

using namespace tvcg;

extern "C" size_t tmc_workspace_size(int order, const int64_t* dims, int mode, int64_t R, tvc_dtype dtype) {
  Shape s;
  if (!valid_dtype(dtype) || R < 1 || make_shape(order, dims, mode, &s) != TVC_OK) return 0;
  return std::max(tmc_plan(s, R, dtype, nullptr, true).ws, tmc_plan(s, R, dtype, nullptr, false).ws);
}

extern "C" tvc_status tmc(const void* A, int order, const int64_t* dims, int mode, const void* X, int64_t R, void* Y,
                          tvc_dtype dtype, const float* slab_scales, double alpha, double beta, void* workspace,
                          size_t ws_bytes, tvc_stream_t stream) {
  if (!valid_dtype(dtype) || !A || !X || !Y || R < 1) return TVC_ERR_INVALID_ARG;
  Shape s;
  tvc_status rc = make_shape(order, dims, mode, &s);
  if (rc != TVC_OK) return rc;
  int64_t uRv;
  if (__builtin_mul_overflow(s.uv, R, &uRv) || uRv >= ((int64_t)1 << 62)) return TVC_ERR_INVALID_ARG;
  if (!aligned(A, elem_size(dtype)) || !aligned(X, vec_size(dtype)) || !aligned(Y, vec_size(dtype)))
    return TVC_ERR_INVALID_ARG;
  const TmcPlan p = tmc_plan(s, R, dtype, A);
  if (p.ws > 0 && (!workspace || ws_bytes < p.ws)) return TVC_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  switch (dtype) {
    case TVC_F64: return run<TVC_F64>(A, s, X, R, Y, slab_scales, alpha, beta, workspace, ws_bytes, p, st);
    case TVC_F32: return run<TVC_F32>(A, s, X, R, Y, slab_scales, alpha, beta, workspace, ws_bytes, p, st);
    case TVC_BF16: return run<TVC_BF16>(A, s, X, R, Y, slab_scales, alpha, beta, workspace, ws_bytes, p, st);
    case TVC_E4M3: return run<TVC_E4M3>(A, s, X, R, Y, slab_scales, alpha, beta, workspace, ws_bytes, p, st);
    case TVC_F16: return run<TVC_F16>(A, s, X, R, Y, slab_scales, alpha, beta, workspace, ws_bytes, p, st);
    case TVC_F32D: return run<TVC_F32D>(A, s, X, R, Y, slab_scales, alpha, beta, workspace, ws_bytes, p, st);
  }
  return TVC_ERR_INVALID_ARG;
}
