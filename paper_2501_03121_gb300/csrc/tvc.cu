// Mode-oblivious dense tensor-vector contraction  Y = alpha (A x_k x) + beta Y
// (Section 3 definition; Eq. 1 form for one process).
//
// The tensor is always streamed from HBM in its own flat (row-major) order,
// whatever k is; only the mapping of loaded elements to outputs changes with
// the matricized view u x n_k x v:
//   * COLS  (v >= 32): one thread owns VEC consecutive outputs (i, l..l+VEC-1)
//           and walks the n_k rows of its slab; a warp reads 32*VEC contiguous
//           elements per row (128-bit loads when alignment allows).  This is
//           the column-block split of the paper's vector-matrix case.
//   * ROWS  (v == 1): a group of G lanes per row (the matrix-vector case,
//           row blocks), 128-bit loads along the row, shuffle reduction.
//   * SLAB  (1 < v < 32, large slabs): one warp per slab; lane (jj, l) reads
//           element l of rows jj, jj+G, ... so each step is one contiguous run
//           of g = v*floor(32/v) elements; lanes with equal l are reduced by
//           shuffles at the end.
//   * TILE  (1 < v < 32, small slabs): a block copies R whole slabs (contiguous)
//           into shared memory and each thread contracts one output from there.
// When the outputs alone cannot fill the GPU, n_k is split over blockIdx.y
// ("split-K"); the partial results go to the workspace and a second kernel
// adds them in a fixed order (deterministic).
#include <algorithm>
#include <mutex>
#include <set>

#include "common.cuh"
#include "internal.h"
#include "tma.cuh"
#include "tvc_args.cuh"

namespace tvcg {

// Sticky device error word of the staged kernels: a bounded wait that gave
// up writes its code here (1: producer waited for a free stage, 2: a
// consumer waited for a tile).  Read and cleared by tvc_device_error().
__device__ int g_tvc_device_error = 0;

constexpr int kThreads = 256;
constexpr int kWarpsPerBlock = kThreads / kWarp;
constexpr int kRB = 64;  // additions per accumulator between folds

// x entries j .. j+VEC-1 (j a multiple of VEC): 16-byte loads when x is
// 16-byte aligned and no per-row slab scale applies (k > 0), else one by one.
template <tvc_dtype DT, int VEC>
__device__ __forceinline__ void xvec(const TvcArgs<DT>& a, int64_t j, float (&xq)[VEC]) {
  const float* x = static_cast<const float*>(a.x);
  const bool fold = kNarrow<DT> && a.mode0 && a.scales;
  if constexpr (VEC % 4 == 0) {
    if (!fold && ((reinterpret_cast<uintptr_t>(x) & 15) == 0)) {
#pragma unroll
      for (int e = 0; e < VEC; e += 4) {
        const float4 f = __ldg(reinterpret_cast<const float4*>(x + j + e));
        xq[e] = f.x;
        xq[e + 1] = f.y;
        xq[e + 2] = f.z;
        xq[e + 3] = f.w;
      }
      return;
    }
  }
#pragma unroll
  for (int e = 0; e < VEC; e++) xq[e] = xval(a, j + e);
}

// ------------------------------------------------------------------ COLS --

template <tvc_dtype DT, int VEC, int DROWS>
__global__ void __launch_bounds__(kThreads) tvc_cols_kernel(const TvcArgs<DT> a) {
  if (skip(a.done)) return;
  using E = Elem<DT>;
  using T = typename E::T;
  const int64_t o = ((int64_t)blockIdx.x * kThreads + threadIdx.x) * VEC;
  if (o >= a.uv) return;
  const int64_t i = div_v(a, o);
  const int64_t l = o - i * a.v;
  const int64_t j0 = (int64_t)blockIdx.y * a.chunk;
  const int64_t j1 = min(a.nk, j0 + a.chunk);
  const int64_t st = a.v;
  const T* p = a.A + (i * a.nk + j0) * st + l;
  int64_t j = j0;
  int blk = 0;
  if constexpr (kF64Acc<DT>) {
    const double* x = static_cast<const double*>(a.x);
    AccF64<VEC> acc;
    acc.init();
    for (; j + 8 <= j1; j += 8) {
      typename E::C r[8][VEC];
#pragma unroll
      for (int q = 0; q < 8; q++) E::template load<VEC>(p + q * st, r[q]);
#pragma unroll
      for (int q = 0; q < 8; q++) {
        if (q < DROWS)
          acc.dfma(r[q], __ldg(x + j + q));
        else
          acc.emul(r[q], x + j + q, ldxs(a.xs + j + q));
      }
      p += 8 * st;
      if (++blk == kRB / 8) {
        acc.fold();
        blk = 0;
      }
    }
    if (j < j1) {  // the last < 8 rows: all loads in flight at once
      typename E::C r[7][VEC];
#pragma unroll
      for (int q = 0; q < 7; q++)
        if (j + q < j1) E::template load<VEC>(p + q * st, r[q]);
#pragma unroll
      for (int q = 0; q < 7; q++)
        if (j + q < j1) acc.emul(r[q], x + j + q, ldxs(a.xs + j + q));
    }
    acc.fold();
#pragma unroll
    for (int e = 0; e < VEC; e++) emit(a, blockIdx.y, o + e, acc.result(e));
  } else {
    AccF32<VEC> acc;
    acc.init();
    for (; j + 8 <= j1; j += 8) {
      float r[8][VEC];
#pragma unroll
      for (int q = 0; q < 8; q++) E::template load<VEC>(p + q * st, r[q]);
#pragma unroll
      for (int q = 0; q < 8; q++) acc.mac(r[q], xval(a, j + q));
      p += 8 * st;
      if (++blk == kRB / 8) {
        acc.fold();
        blk = 0;
      }
    }
    for (; j < j1; j++, p += st) {
      float r[VEC];
      E::template load<VEC>(p, r);
      acc.mac(r, xval(a, j));
    }
    acc.fold();
    const float sc = out_scale(a, i);
#pragma unroll
    for (int e = 0; e < VEC; e++) emit(a, blockIdx.y, o + e, __fmul_rn(acc.result(e), sc));
  }
}

// Columns with a per-thread asynchronous pipeline (narrow storage): each
// thread keeps the next D rows of its 16-byte column piece in flight with
// cp.async (global -> its own shared-memory slots, no registers held), and
// consumes row j while row j + D is being fetched.  Each thread waits only
// for its own copies (cp.async.wait_group), so no block barrier is needed.
// This keeps D * 16 bytes per thread in flight, which the register-bound
// column kernel cannot for 8- or 16-element vectors.
constexpr int kAsyncDepth = 12;


template <tvc_dtype DT, int VEC>
__global__ void __launch_bounds__(kThreads) tvc_cols_async_kernel(const TvcArgs<DT> a) {
  if (skip(a.done)) return;
  using E = Elem<DT>;
  using T = typename E::T;
  static_assert(VEC * sizeof(T) == 16, "16-byte column pieces");
  __shared__ __align__(16) uint4 stage[kAsyncDepth][kThreads];
  const int64_t o = ((int64_t)blockIdx.x * kThreads + threadIdx.x) * VEC;
  const bool active = o < a.uv;
  const int64_t oo = active ? o : 0;
  const int64_t i = div_v(a, oo);
  const int64_t l = oo - i * a.v;
  const int64_t j0 = (int64_t)blockIdx.y * a.chunk;
  const int64_t j1 = min(a.nk, j0 + a.chunk);
  const int64_t st = a.v;
  const T* p = a.A + (i * a.nk + j0) * st + l;
  const int64_t n = active ? (j1 - j0) : 0;
#pragma unroll
  for (int d = 0; d < kAsyncDepth; d++) {
    if (d < n) cp_async16(&stage[d][threadIdx.x], p + d * st);
    cp_async_commit();
  }
  AccF32<VEC> acc;
  acc.init();
  int blk = 0;
  int slot = 0;
  for (int64_t r = 0; r < n; r++) {
    cp_async_wait<kAsyncDepth - 1>();
    float v[VEC];
    E::template load<VEC, true>(reinterpret_cast<const T*>(&stage[slot][threadIdx.x]), v);
    const float xv = xval(a, j0 + r);
    // the slot is free again: fetch row r + D into it
    if (r + kAsyncDepth < n) cp_async16(&stage[slot][threadIdx.x], p + (r + kAsyncDepth) * st);
    cp_async_commit();
    acc.mac(v, xv);
    if (++slot == kAsyncDepth) slot = 0;
    if (++blk == kRB) {
      acc.fold();
      blk = 0;
    }
  }
  cp_async_wait<0>();
  if (!active) return;
  acc.fold();
  const float sc = out_scale(a, i);
#pragma unroll
  for (int e = 0; e < VEC; e++) emit(a, blockIdx.y, o + e, __fmul_rn(acc.result(e), sc));
}

// ------------------------------------------------------------------ ROWS --

template <class V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
  return v;
}

// Rows of the matrix-vector case (v == 1): a group of G lanes (G a power of
// two <= 32) owns one row segment; lane p of the group loads VEC consecutive
// elements at p*VEC + step*G*VEC, so a warp reads 32/G rows at once, each
// as one contiguous run per step.  The group's partial sums are reduced by
// xor-shuffles; for FP64 the float-float pairs are reduced in FP32 with
// TwoSum, so the reduction stays off the FP64 pipe.
// SH: FP64 pairs of rows of odd length (see below); a separate instance, so
// that the even rows keep their register count (48; 62 with the shift logic
// cost them 20% of the resident warps and 10% of their speed).
template <tvc_dtype DT, int VEC, int G, bool SH = false>
__global__ void __launch_bounds__(kThreads) tvc_rows_kernel(const TvcArgs<DT> a) {
  if (skip(a.done)) return;
  using E = Elem<DT>;
  using T = typename E::T;
  constexpr int STEP = G * VEC;
  constexpr int UNR = 4;
  constexpr int RPW = kWarp / G;  // rows per warp
  const int lane = threadIdx.x & (kWarp - 1);
  const int p = lane & (G - 1);
  const int64_t row = ((int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5)) * RPW + lane / G;
  const bool active = row < a.u;
  const int64_t j0 = (int64_t)blockIdx.y * a.chunk;
  const int64_t j1 = min(a.nk, j0 + a.chunk);
  const T* rp = a.A + (active ? row : 0) * a.nk;
  // FP64 pairs (VEC == 2) of a row whose segment starts 8 bytes past a
  // 16-byte boundary (odd n_k): its first element goes alone and the pairs
  // start one element later, against the shifted split x (xs1).
  int sh = 0;
  int64_t jb = j0;
  if constexpr (SH) {
    sh = (int)(((active ? row : 0) * a.nk + j0) & 1);
    jb = j0 + sh;
  }
  const int64_t ngroups = active ? (j1 - jb) / (UNR * STEP) : 0;
  const int64_t jt0 = jb + ngroups * UNR * STEP;  // start of the ragged tail
  int64_t j = jb + p * VEC;
  int blk = 0;
  if constexpr (kF64Acc<DT>) {
    const double* x = static_cast<const double*>(a.x);
    AccF64<VEC> acc;
    acc.init();
    const XSplit* const xsp = SH && sh ? a.xs1 + 1 : a.xs;  // pieces of (jq, jq + 1) at xsp + jq, 16-byte aligned
    if constexpr (SH) {
      if (sh && active && p == 0 && j0 < j1) {
        typename E::C r[1];
        E::template load<1>(rp + j0, r);
        acc.emul1(0, r[0], x + j0, ldxs(a.xs + j0));
      }
    }
    // kRB / UNR groups per fold.  With 8-byte loads (VEC == 1) the fold sits
    // outside the inner loop: a fold test per group is if-converted there
    // into masked FP64 work on every group (measured: 30623-element rows
    // 4.1 -> 5.1 TB/s); with 16-byte loads the per-group test measured
    // faster (65536 x 16384: 6.7 vs 6.2 TB/s).
    constexpr int64_t kGroupsPerFold = (VEC == 1) ? kRB / UNR : 1;
    for (int64_t g0 = 0; g0 < ngroups; g0 += kGroupsPerFold) {
      const int64_t g1 = min(ngroups, g0 + kGroupsPerFold);
      for (int64_t g = g0; g < g1; g++, j += UNR * STEP) {
        typename E::C r[UNR][VEC];
#pragma unroll
        for (int q = 0; q < UNR; q++) E::template load<VEC>(rp + j + q * STEP, r[q]);
#pragma unroll
        for (int q = 0; q < UNR; q++) {
          const int64_t jq = j + q * STEP;
          if constexpr (VEC == 2) {
            float4 s2 = __ldg(reinterpret_cast<const float4*>(xsp + jq));
            acc.emul1(0, r[q][0], x + jq, XSplit{s2.x, s2.y});
            acc.emul1(1, r[q][1], x + jq + 1, XSplit{s2.z, s2.w});
          } else {
#pragma unroll
            for (int e = 0; e < VEC; e++) acc.emul1(e, r[q][e], x + jq + e, ldxs(a.xs + jq + e));
          }
        }
      }
      if constexpr (VEC == 1) {
        acc.fold();
      } else if (++blk == kRB / UNR) {
        acc.fold();
        blk = 0;
      }
    }
    if (active)
      for (int64_t jj = jt0 + p; jj < j1; jj += G) {
        typename E::C r[1];
        E::template load<1>(rp + jj, r);
        acc.emul1(0, r[0], x + jj, ldxs(a.xs + jj));
      }
    // Combine the VEC columns of the lane into pair 0 (and total d).
    float s = acc.s[0], c = acc.c[0];
    double d = acc.d[0];
#pragma unroll
    for (int e = 1; e < VEC; e++) {
      float t, err;
      two_sum(s, acc.s[e], t, err);
      s = t;
      c = __fadd_rn(c, __fadd_rn(acc.c[e], err));
      d += acc.d[e];
    }
    const bool need_d = __any_sync(0xFFFFFFFFu, d != 0.0);
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
      const float s2 = __shfl_xor_sync(0xFFFFFFFFu, s, off);
      const float c2 = __shfl_xor_sync(0xFFFFFFFFu, c, off);
      float t, err;
      two_sum(s, s2, t, err);
      s = t;
      c = __fadd_rn(c, __fadd_rn(c2, err));
    }
    if (need_d) {
#pragma unroll
      for (int off = G / 2; off > 0; off >>= 1) d += __shfl_xor_sync(0xFFFFFFFFu, d, off);
    }
    if (active && p == 0) emit(a, blockIdx.y, row, (d + (double)s) + (double)c);
  } else {
    AccF32<VEC> acc;
    acc.init();
    for (int64_t g = 0; g < ngroups; g++, j += UNR * STEP) {
      float r[UNR][VEC];
#pragma unroll
      for (int q = 0; q < UNR; q++) E::template load<VEC>(rp + j + q * STEP, r[q]);
#pragma unroll
      for (int q = 0; q < UNR; q++) {
        float xq[VEC];
        xvec<DT, VEC>(a, j + q * STEP, xq);
#pragma unroll
        for (int e = 0; e < VEC; e++) acc.a[e] = __fmaf_rn(r[q][e], xq[e], acc.a[e]);
      }
      if (++blk == kRB / UNR) {
        acc.fold();
        blk = 0;
      }
    }
    if (active)
      for (int64_t jj = jt0 + p; jj < j1; jj += G) {
        float r[1];
        E::template load<1>(rp + jj, r);
        acc.a[0] = __fmaf_rn(r[0], xval(a, jj), acc.a[0]);
      }
    acc.fold();
    float tot = 0.0f;
#pragma unroll
    for (int e = 0; e < VEC; e++) tot += acc.result(e);
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) tot += __shfl_xor_sync(0xFFFFFFFFu, tot, off);
    if (active && p == 0) emit(a, blockIdx.y, row, __fmul_rn(tot, out_scale(a, row)));
  }
}

// Long rows of the FP32/BF16/E4M3 types (v == 1): the whole warp walks RB
// consecutive rows together, lane p taking VEC elements at p*VEC + step*32*VEC
// of each, so that every piece of x held in registers serves RB rows.  With
// one row per lane group (tvc_rows_kernel) the FP32 x is read through L1 at
// s_x/s_A times the rate of A (4x for E4M3 codes, 2x for BF16), which held
// the narrow long rows far below the HBM rate.  Each row keeps two FP32
// accumulators, folded into a compensated sum every 64 products.
template <tvc_dtype DT, int VEC, int RB, int UNR>
__global__ void __launch_bounds__(kThreads) tvc_rows_multi_kernel(const TvcArgs<DT> a) {
  static_assert(!kF64Acc<DT>, "FP64 arithmetic rows use the float-float kernels");
  static_assert(VEC * sizeof(typename Elem<DT>::T) == 16, "16-byte pieces");
  if (skip(a.done)) return;
  using E = Elem<DT>;
  using T = typename E::T;
  constexpr int STEP = kWarp * VEC;
  constexpr int FOLD = (2 * kRB / VEC) / UNR;  // groups between folds
  static_assert(FOLD >= 1, "fold interval");
  const int lane = threadIdx.x & (kWarp - 1);
  const int64_t row0 = ((int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5)) * RB;
  if (row0 >= a.u) return;  // warp-uniform; no block-wide barrier follows
  const int64_t j0 = (int64_t)blockIdx.y * a.chunk;
  const int64_t j1 = min(a.nk, j0 + a.chunk);
  const int nr = (int)min((int64_t)RB, a.u - row0);  // rows of this warp (warp-uniform)
  const T* rp[RB];
#pragma unroll
  for (int r = 0; r < RB; r++) rp[r] = a.A + min(row0 + r, a.u - 1) * a.nk;
  float acc[RB][2];
  KahanF32 tot[RB];
#pragma unroll
  for (int r = 0; r < RB; r++) acc[r][0] = acc[r][1] = 0.0f;
  auto fold = [&]() {
#pragma unroll
    for (int r = 0; r < RB; r++) {
      tot[r].add(acc[r][0]);
      tot[r].add(acc[r][1]);
      acc[r][0] = acc[r][1] = 0.0f;
    }
  };
  const int64_t ngroups = (j1 - j0) / (UNR * STEP);
  int64_t j = j0 + lane * VEC;
  int blk = 0;
  for (int64_t g = 0; g < ngroups; g++, j += UNR * STEP) {
    uint4 w[UNR][RB];  // packed codes, decoded where they are used
#pragma unroll
    for (int q = 0; q < UNR; q++)
#pragma unroll
      for (int r = 0; r < RB; r++) w[q][r] = (r < nr) ? ld_stream<16>(rp[r] + j + q * STEP).v : make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int q = 0; q < UNR; q++) {
      float xq[VEC];
      xvec<DT, VEC>(a, j + q * STEP, xq);
#pragma unroll
      for (int r = 0; r < RB; r++) {
        float v[VEC];
        E::decode16(w[q][r], v);
#pragma unroll
        for (int e = 0; e < VEC; e++) acc[r][e & 1] = __fmaf_rn(v[e], xq[e], acc[r][e & 1]);
      }
    }
    if (++blk == FOLD) {
      fold();
      blk = 0;
    }
  }
  // Tail of fewer than UNR steps: (j1 - j0) is a multiple of VEC (the planner
  // takes VEC dividing n_k and a chunk that is a multiple of 32*VEC).
  for (; j < j1; j += STEP) {
    float xq[VEC];
    xvec<DT, VEC>(a, j, xq);
#pragma unroll
    for (int r = 0; r < RB; r++) {
      if (r < nr) {
        float v[VEC];
        E::template load<VEC>(rp[r] + j, v);
#pragma unroll
        for (int e = 0; e < VEC; e++) acc[r][e & 1] = __fmaf_rn(v[e], xq[e], acc[r][e & 1]);
      }
    }
  }
  fold();
  float mine = 0.0f;
#pragma unroll
  for (int r = 0; r < RB; r++) {
    const float t = warp_sum(tot[r].value());
    if (lane == r) mine = t;
  }
  if (lane < RB && row0 + lane < a.u) emit(a, blockIdx.y, row0 + lane, __fmul_rn(mine, out_scale(a, row0 + lane)));
}

// FP64 rows with G < 32 lanes per row (short rows): each warp takes 32 rows
// in G passes of 32/G rows, keeps every finished row in a per-lane slot
// (lane L holds row L of the warp), and converts and stores the 32 results
// with full-warp FP64 instructions.  The FP64 pipe takes a warp instruction
// at the same cost whatever its active mask, so converting per pass would
// spend it G times over.  Products and reductions stay on the FP32 pipe.
template <tvc_dtype DT, int VEC, int G, int DQ>
__global__ void __launch_bounds__(kThreads) tvc_rows_f64_slots_kernel(const TvcArgs<DT> a) {
  if (skip(a.done)) return;
  static_assert(kF64Acc<DT>, "FP64 arithmetic");
  using E = Elem<DT>;
  using T = typename E::T;
  constexpr int STEP = G * VEC;
  constexpr int GPW = kWarp / G;
  constexpr int UNR = (VEC == 1) ? 8 : 4;  // 8-byte loads: more of them in flight
  const int lane = threadIdx.x & (kWarp - 1);
  const int p = lane & (G - 1);
  const int gw = lane / G;
  const int64_t wrow0 = ((int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5)) * kWarp;
  if (wrow0 >= a.u) return;  // whole warp
  const int64_t j0 = (int64_t)blockIdx.y * a.chunk;
  const int64_t j1 = min(a.nk, j0 + a.chunk);
  const double* x = static_cast<const double*>(a.x);
  float slot_s = 0.0f, slot_c = 0.0f;
  double slot_d = 0.0;
  for (int it = 0; it < G; it++) {
    const int64_t row = wrow0 + it * GPW + gw;
    const bool active = row < a.u;
    const T* rp = a.A + (active ? row : 0) * a.nk;
    float sacc = 0.0f, cacc = 0.0f;
    double d = 0.0;
    // 8-byte loads (VEC == 1): branch-free steps (df_step) with the window
    // bits in `bad`, redone with DFMA when set (measured 1.1-1.2x on odd
    // rows); 16-byte loads keep df_mac's branch, which measured faster there
    // (fewer registers, more warps in flight).
    uint32_t bad = 0;
    if (active && VEC == 1) {
      // 8-byte loads: every pass issues all its loads before the products,
      // the last (partial) pass too; steps past the row end are neither
      // loaded nor multiplied (j1 - j0 is a multiple of VEC).  (Measured on
      // odd rows of 63 .. 979 elements: 1.3-1.8x; with 16-byte loads the
      // unpredicated loop below measured faster.)
      for (int64_t jj = j0 + p * VEC; jj < j1; jj += UNR * STEP) {
        typename E::C r[UNR][VEC];
#pragma unroll
        for (int q = 0; q < UNR; q++)
          if (jj + q * STEP < j1) E::template load<VEC>(rp + jj + q * STEP, r[q]);
#pragma unroll
        for (int q = 0; q < UNR; q++) {
          if (jj + q * STEP >= j1) break;
#pragma unroll
          for (int e = 0; e < VEC; e++) {
            if (q < DQ)  // this share of the steps runs on the FP64 pipe
              d = fma((double)r[q][e], __ldg(x + jj + q * STEP + e), d);
            else
              df_step(sacc, cacc, bad, r[q][e], ldxs(a.xs + jj + q * STEP + e));
          }
        }
      }
    } else if (active) {
      int64_t jj = j0 + p * VEC;
      for (; jj + (UNR - 1) * STEP + VEC <= j1; jj += UNR * STEP) {
        typename E::C r[UNR][VEC];
#pragma unroll
        for (int q = 0; q < UNR; q++) E::template load<VEC>(rp + jj + q * STEP, r[q]);
#pragma unroll
        for (int q = 0; q < UNR; q++)
#pragma unroll
          for (int e = 0; e < VEC; e++) {
            if (q < DQ)
              d = fma((double)r[q][e], __ldg(x + jj + q * STEP + e), d);
            else
              df_mac(sacc, cacc, d, r[q][e], x + jj + q * STEP + e, ldxs(a.xs + jj + q * STEP + e));
          }
      }
      for (; jj + VEC <= j1; jj += STEP) {
        typename E::C r[VEC];
        E::template load<VEC>(rp + jj, r);
#pragma unroll
        for (int e = 0; e < VEC; e++) df_mac(sacc, cacc, d, r[e], x + jj + e, ldxs(a.xs + jj + e));
      }
    }
    if (VEC == 1 && active && (bad != 0 || sacc != sacc || cacc != cacc)) {
      // rare: this lane's part of the row again, exactly, on the DFMA pipe
      sacc = 0.0f;
      cacc = 0.0f;
      d = 0.0;
      for (int64_t jj = j0 + p * VEC; jj < j1; jj += STEP)
#pragma unroll
        for (int e = 0; e < VEC; e++) d = fma((double)rp[jj + e], x[jj + e], d);
    }
    if (DQ > 0 && df_out_of_window(d) == 0) {  // fold the DFMA share into the pair
      df_add_double(sacc, cacc, d);
      d = 0.0;
    }
    const bool anyd = __any_sync(0xFFFFFFFFu, __double_as_longlong(d) != 0);
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
      const float s2 = __shfl_xor_sync(0xFFFFFFFFu, sacc, off);
      const float c2 = __shfl_xor_sync(0xFFFFFFFFu, cacc, off);
      float t, err;
      two_sum(sacc, s2, t, err);
      sacc = t;
      cacc = __fadd_rn(cacc, __fadd_rn(c2, err));
    }
    if (anyd) {
#pragma unroll
      for (int off = G / 2; off > 0; off >>= 1) d += __shfl_xor_sync(0xFFFFFFFFu, d, off);
    }
    // lanes it*GPW .. it*GPW + GPW - 1 take the rows of this pass
    const int rel = lane - it * GPW;
    const bool mine = rel >= 0 && rel < GPW;
    const int srcl = mine ? rel * G : 0;
    const float ss = __shfl_sync(0xFFFFFFFFu, sacc, srcl);
    const float cc = __shfl_sync(0xFFFFFFFFu, cacc, srcl);
    if (mine) {
      slot_s = ss;
      slot_c = cc;
    }
    if (anyd) {
      const double dd = __shfl_sync(0xFFFFFFFFu, d, srcl);
      if (mine) slot_d = dd;
    }
  }
  const int64_t row = wrow0 + lane;
  if (row < a.u) emit(a, blockIdx.y, row, (slot_d + (double)slot_s) + (double)slot_c);
}

// Short rows (v == 1, n_k <= NST*G*VEC): a group of G lanes (runtime, power
// of two <= 32) owns B rows per iteration; lane p covers the NST steps
// j = p*VEC + q*G*VEC of each.  Those positions are the same in every row,
// so each lane keeps its pieces of x in registers while the groups walk the
// rows persistently (grid-stride).  All B*NST loads of an iteration are
// issued before any arithmetic, which keeps enough bytes in flight.
template <tvc_dtype DT, int VEC, int NST>
__global__ void __launch_bounds__(kThreads) tvc_rows_short_kernel(const TvcArgs<DT> a, int G) {
  if (skip(a.done)) return;
  // Rows per group per iteration: about 32 elements of loads per lane.
  constexpr int B = (32 / (NST * VEC)) < 1 ? 1 : ((32 / (NST * VEC)) > 4 ? 4 : (32 / (NST * VEC)));
  using E = Elem<DT>;
  using T = typename E::T;
  using Cm = typename E::C;
  const int lane = threadIdx.x & (kWarp - 1);
  const int p = lane & (G - 1);
  const int rpw = kWarp / G;
  const int64_t warp_row0 = ((int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5)) * rpw * B;
  const int64_t rows_per_iter = (int64_t)gridDim.x * kWarpsPerBlock * rpw * B;
  const int nk = (int)a.nk;
  const int step = G * VEC;
  float xh[NST][VEC], xl[NST][VEC];
#pragma unroll
  for (int q = 0; q < NST; q++)
#pragma unroll
    for (int e = 0; e < VEC; e++) {
      const int j = p * VEC + q * step + e;
      if constexpr (kF64Acc<DT>) {
        XSplit t = (j < nk) ? ldxs(a.xs + j) : XSplit{0.0f, 0.0f};
        xh[q][e] = t.xh;
        xl[q][e] = t.xl;
      } else {
        xh[q][e] = (j < nk) ? xval(a, j) : 0.0f;
        xl[q][e] = 0.0f;
      }
    }
  // Row b of the warp's iteration: wr + b*rpw + lane/G.
  for (int64_t wr = warp_row0; wr < a.u; wr += rows_per_iter) {
    Cm r[B][NST][VEC];
#pragma unroll
    for (int b = 0; b < B; b++) {
      const int64_t row = wr + (int64_t)b * rpw + lane / G;
      const T* rp = a.A + row * a.nk;
#pragma unroll
      for (int q = 0; q < NST; q++) {
        const int j = p * VEC + q * step;
        if (row < a.u && j < nk) {
          E::template load<VEC>(rp + j, r[b][q]);
        } else {
#pragma unroll
          for (int e = 0; e < VEC; e++) r[b][q][e] = (Cm)0;
        }
      }
    }
    if constexpr (kF64Acc<DT>) {
      const double* x = static_cast<const double*>(a.x);
      float sb[B], cb[B];
      double db[B];
      bool anyd = false;
#pragma unroll
      for (int b = 0; b < B; b++) {
        const int64_t row = wr + (int64_t)b * rpw + lane / G;
        float s = 0.0f, c = 0.0f;
        double d = 0.0;
#pragma unroll
        for (int q = 0; q < NST; q++) {
          // Skip padding (past the row or past the last row): a zero would
          // take the out-of-window path.
          if (row < a.u && p * VEC + q * step < nk) {
#pragma unroll
            for (int e = 0; e < VEC; e++)
              df_mac(s, c, d, r[b][q][e], x + (p * VEC + q * step + e), XSplit{xh[q][e], xl[q][e]});
          }
        }
        sb[b] = s;
        cb[b] = c;
        db[b] = d;
        anyd |= (__double_as_longlong(d) != 0);  // integer test: no FP64 pipe
      }
      // Group reductions of the B rows (independent, so they interleave).
      for (int off = G / 2; off > 0; off >>= 1) {
#pragma unroll
        for (int b = 0; b < B; b++) {
          const float s2 = __shfl_xor_sync(0xFFFFFFFFu, sb[b], off);
          const float c2 = __shfl_xor_sync(0xFFFFFFFFu, cb[b], off);
          float t, err;
          two_sum(sb[b], s2, t, err);
          sb[b] = t;
          cb[b] = __fadd_rn(cb[b], __fadd_rn(c2, err));
        }
      }
      if (__any_sync(0xFFFFFFFFu, anyd)) {
        for (int off = G / 2; off > 0; off >>= 1) {
#pragma unroll
          for (int b = 0; b < B; b++) db[b] += __shfl_xor_sync(0xFFFFFFFFu, db[b], off);
        }
      }
      // Epilogue: every lane of a group holds the B results; lane p takes
      // rows b = p, p + G, ... (picked with selects, not register indexing),
      // so one FP64 conversion serves up to B rows per group.
      for (int b0 = 0; b0 < B; b0 += G) {
        const int bsel = b0 + p;
        float s = 0.0f, c = 0.0f;
        double d = 0.0;
#pragma unroll
        for (int b = 0; b < B; b++)
          if (b == bsel) {
            s = sb[b];
            c = cb[b];
            d = db[b];
          }
        const int64_t row = wr + (int64_t)bsel * rpw + lane / G;
        if (bsel < B && row < a.u) emit(a, 0, row, (d + (double)s) + (double)c);
      }
    } else {
#pragma unroll
    for (int b = 0; b < B; b++) {
      const int64_t row = wr + (int64_t)b * rpw + lane / G;
      {
        float acc = 0.0f;
#pragma unroll
        for (int q = 0; q < NST; q++)
#pragma unroll
          for (int e = 0; e < VEC; e++) acc = __fmaf_rn(r[b][q][e], xh[q][e], acc);
        for (int off = G / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
        if (row < a.u && p == 0) emit(a, 0, row, __fmul_rn(acc, out_scale(a, row)));
      }
    }
    }
  }
}

// Staged rows (v == 1, n_k <= nst*G*VEC): the matrix-vector case with short
// rows, fed by the TMA engine.  One producer lane copies tiles of R whole
// rows (contiguous, R*n_k elements) into an S-stage ring of shared memory
// with cp.async.bulk; eight consumer warps reduce the rows of each tile from
// shared memory (a group of G lanes per row, the lane's pieces of x kept in
// registers), then each warp converts and stores its RW rows with one
// coalesced store per lane.  Full/empty mbarriers order the ring; every wait
// is bounded (tma.cuh).  A ragged last tile (byte count not a multiple of
// 16) is read by the consumers straight from global memory.
// A tile goes through the copy engine only when its source address and size
// are multiples of 16 bytes (the stage buffers are 16-byte aligned: the
// planner makes the tile size a multiple of 16); otherwise the consumers
// read it from global memory.  Producer and consumers decide alike.
template <class T>
__device__ __forceinline__ bool tile_by_copy(const T* src, uint64_t bytes) {
  return ((bytes & 15) == 0) && ((reinterpret_cast<uintptr_t>(src) & 15) == 0);
}

struct RowsTmaParams {
  int R, RW, S, G, nst, dq;  // dq: steps per lane sent to the DFMA pipe (FP64)
  int64_t ntiles;
  uint32_t tile_bytes;
};

constexpr int kTmaConsumerWarps = 8;
constexpr int kTmaThreads = (kTmaConsumerWarps + 1) * kWarp;

template <tvc_dtype DT, int VEC, int NST>
__global__ void __launch_bounds__(kTmaThreads, 2) tvc_rows_tma_kernel(const TvcArgs<DT> a, RowsTmaParams prm) {
  if (skip(a.done)) return;
  using E = Elem<DT>;
  using T = typename E::T;
  using Cm = typename E::C;
  extern __shared__ __align__(128) unsigned char smraw[];
  const int S = prm.S, R = prm.R, RW = prm.RW;
  unsigned char* stages = smraw;
  size_t off = (size_t)S * prm.tile_bytes;
  float2* wres = reinterpret_cast<float2*>(smraw + off);  // [warps][RW]
  off += (size_t)kTmaConsumerWarps * RW * sizeof(float2);
  off += (size_t)kTmaConsumerWarps * RW * sizeof(double);  // [warps][RW] doubles, part of the host's layout
  uint64_t* full = reinterpret_cast<uint64_t*>(smraw + off);
  uint64_t* empty = full + S;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int q = 0; q < S; q++) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], kTmaConsumerWarps);
    }
    mbar_fence_init();
  }
  __syncthreads();
  const int nk = (int)a.nk;
  if (warp == kTmaConsumerWarps) {  // producer warp
    if (lane == 0) {
      int k = 0;
      for (int64_t t = blockIdx.x; t < prm.ntiles; t += gridDim.x, k++) {
        const int st = k % S;
        if (k >= S && !mbar_wait(&empty[st], ((k / S) - 1) & 1, &g_tvc_device_error, 1)) break;
        const int64_t rows = min((int64_t)R, a.u - t * R);
        const uint64_t bytes = (uint64_t)rows * nk * sizeof(T);
        if (tile_by_copy(a.A + t * R * a.nk, bytes)) {
          mbar_arrive_expect_tx(&full[st], (uint32_t)bytes);
          tma_load_1d(stages + (size_t)st * prm.tile_bytes, a.A + t * R * a.nk, (uint32_t)bytes, &full[st]);
        } else {
          mbar_arrive(&full[st]);
        }
      }
      // Never leave with copies in flight: wait (bounded) for the last
      // phases issued on every stage.
      for (int q = 0; q < S && q < k; q++) {
        const int kk = k - 1 - q;
        mbar_wait(&full[kk % S], (kk / S) & 1, &g_tvc_device_error, 3, 400000000LL);
      }
    }
    return;
  }
  const int G = prm.G;
  const int p = lane & (G - 1);
  const int gpw = kWarp / G;               // groups per warp
  const int gw = lane / G;                 // group within the warp
  const int step = G * VEC;
  float xh[NST][VEC], xl[NST][VEC];
  bool x_in_window = true;  // every x piece of this lane can take the fast path
#pragma unroll
  for (int q = 0; q < NST; q++)
#pragma unroll
    for (int e = 0; e < VEC; e++) {
      const int j = p * VEC + q * step + e;
      const bool ok = q < prm.nst && j < nk;
      if constexpr (kF64Acc<DT>) {
        XSplit t = ok ? ldxs(a.xs + j) : XSplit{0.0f, 0.0f};
        xh[q][e] = t.xh;
        xl[q][e] = t.xl;
        if (!(t.xh == t.xh)) x_in_window = false;
      } else {
        xh[q][e] = ok ? xval(a, j) : 0.0f;
        xl[q][e] = 0.0f;
      }
    }
  float2* myres = wres + warp * RW;
  // FP64: finished rows wait in per-lane slots (lane L holds slot L) until
  // 32 have gathered, so that the FP64 conversions and stores run on full
  // warps (the FP64 pipe takes a warp instruction at the same cost whatever
  // its active mask).
  float slot_s = 0.0f, slot_c = 0.0f;
  double slot_d = 0.0;
  int64_t slot_row = -1;
  int nslot = 0;
  auto flush = [&]() {
    if constexpr (kF64Acc<DT>) {
      if (lane < nslot && slot_row >= 0) emit(a, 0, slot_row, (slot_d + (double)slot_s) + (double)slot_c);
      slot_row = -1;
      nslot = 0;
    }
  };
  int k = 0;
  for (int64_t t = blockIdx.x; t < prm.ntiles; t += gridDim.x, k++) {
    const int st = k % S;
    if (!mbar_wait(&full[st], (k / S) & 1, &g_tvc_device_error, 2)) break;
    const int64_t row0 = t * R;
    const int64_t rows = min((int64_t)R, a.u - row0);
    const uint64_t bytes = (uint64_t)rows * nk * sizeof(T);
    const T* src = tile_by_copy(a.A + row0 * a.nk, bytes)
                       ? reinterpret_cast<const T*>(stages + (size_t)st * prm.tile_bytes)
                       : a.A + row0 * a.nk;
    // rows of this warp: warp*RW .. warp*RW + RW-1; group gw takes every gpw-th
    for (int lr = gw; lr < RW; lr += gpw) {
      const int r = warp * RW + lr;
      const bool active = r < rows;
      const T* rp = src + (int64_t)(active ? r : 0) * nk;
      Cm v[NST][VEC];
#pragma unroll
      for (int q = 0; q < NST; q++) {
        const int j = p * VEC + q * step;
        if (active && q < prm.nst && j < nk) {
          E::template load<VEC, true>(rp + j, v[q]);
        } else {
#pragma unroll
          for (int e = 0; e < VEC; e++) v[q][e] = (Cm)0;
        }
      }
      if constexpr (kF64Acc<DT>) {
        const double* x = static_cast<const double*>(a.x);
        float sacc = 0.0f, cacc = 0.0f;
        double d = 0.0;
        // One warp vote decides between the branch-free path (every element
        // and x piece in the split window) and the checked one.
        uint32_t bad = x_in_window ? 0u : 1u;
#pragma unroll
        for (int q = 0; q < NST; q++)
          if (active && q < prm.nst && p * VEC + q * step < nk) {
#pragma unroll
            for (int e = 0; e < VEC; e++) bad |= df_out_of_window(v[q][e]);
          }
        if (!__any_sync(0xFFFFFFFFu, bad != 0)) {
          // The first dq steps go to the FP64 pipe, the rest to the FP32
          // pipe in float-float arithmetic: both pipes share the work.
#pragma unroll
          for (int q = 0; q < NST; q++) {
            if (active && q < prm.nst && p * VEC + q * step < nk) {
              if (q < prm.dq) {
#pragma unroll
                for (int e = 0; e < VEC; e++) d = fma((double)v[q][e], x[p * VEC + q * step + e], d);
              } else {
#pragma unroll
                for (int e = 0; e < VEC; e++) df_mac_fast(sacc, cacc, v[q][e], XSplit{xh[q][e], xl[q][e]});
              }
            }
          }
        } else {
#pragma unroll
          for (int q = 0; q < NST; q++) {
            if (active && q < prm.nst && p * VEC + q * step < nk) {
#pragma unroll
              for (int e = 0; e < VEC; e++)
                df_mac(sacc, cacc, d, v[q][e], x + (p * VEC + q * step + e), XSplit{xh[q][e], xl[q][e]});
            }
          }
        }
        // The FP64 partial (DFMA share, out-of-window elements) joins the
        // float-float pair before the group reduction when it fits the
        // split window; otherwise (huge or tiny values) it stays FP64 and is
        // reduced on its own (rare: a warp vote).
        double drest = 0.0;
        if (df_out_of_window(d) == 0)
          df_add_double(sacc, cacc, d);
        else
          drest = d;
        const bool anyd = __any_sync(0xFFFFFFFFu, __double_as_longlong(drest) != 0);
        for (int o = G / 2; o > 0; o >>= 1) {
          const float s2 = __shfl_xor_sync(0xFFFFFFFFu, sacc, o);
          const float c2 = __shfl_xor_sync(0xFFFFFFFFu, cacc, o);
          float tt, err;
          two_sum(sacc, s2, tt, err);
          sacc = tt;
          cacc = __fadd_rn(cacc, __fadd_rn(c2, err));
        }
        if (anyd)
          for (int o = G / 2; o > 0; o >>= 1) drest += __shfl_xor_sync(0xFFFFFFFFu, drest, o);
        // Move the gpw finished rows (lanes 0, G, 2G, ...) into slots
        // nslot .. nslot+gpw-1 (nslot is a multiple of gpw).
        const int rel = lane - nslot;
        const int srcl = (rel >= 0 && rel < gpw) ? rel * G : 0;
        const float ss = __shfl_sync(0xFFFFFFFFu, sacc, srcl);
        const float cc = __shfl_sync(0xFFFFFFFFu, cacc, srcl);
        double dd = 0.0;
        if (anyd) dd = __shfl_sync(0xFFFFFFFFu, drest, srcl);
        if (rel >= 0 && rel < gpw) {
          const int rr = warp * RW + (lr - gw) + rel;  // the row group `rel` computed
          slot_s = ss;
          slot_c = cc;
          slot_d = dd;
          slot_row = (rr < rows) ? row0 + rr : -1;
        }
        nslot += gpw;
        if (nslot == kWarp) flush();
      } else {
        float acc = 0.0f;
#pragma unroll
        for (int q = 0; q < NST; q++)
#pragma unroll
          for (int e = 0; e < VEC; e++) acc = __fmaf_rn(v[q][e], xh[q][e], acc);
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if (p == 0) myres[lr] = make_float2(acc, 0.0f);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
    if constexpr (!kF64Acc<DT>) {
      // One coalesced store per lane for the warp's rows.
      for (int lr = lane; lr < RW; lr += kWarp) {
        const int64_t row = row0 + warp * RW + lr;
        if (warp * RW + lr < rows) emit(a, 0, row, __fmul_rn(myres[lr].x, out_scale(a, row)));
      }
      __syncwarp();
    }
  }
  flush();
}

// ------------------------------------------------------------------ SLAB --

template <tvc_dtype DT, int UNR>
__global__ void __launch_bounds__(kThreads) tvc_slab_kernel(const TvcArgs<DT> a, int g, int G) {
  if (skip(a.done)) return;
  using E = Elem<DT>;
  using T = typename E::T;
  using V = typename E::V;
  const int lane = threadIdx.x & (kWarp - 1);
  const int64_t slab = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (slab >= a.u) return;
  const int64_t j0 = (int64_t)blockIdx.y * a.chunk;
  const int64_t j1 = min(a.nk, j0 + a.chunk);
  const int l = lane % (int)a.v;
  const int jj = lane / (int)a.v;
  const bool active = lane < g;
  const int64_t st = (int64_t)G * a.v;
  const T* p = a.A + (slab * a.nk + j0 + jj) * a.v + l;
  V tot;
  if constexpr (kF64Acc<DT>) {
    const double* x = static_cast<const double*>(a.x);
    AccF64<1> acc;
    acc.init();
    if (active) {
      int64_t j = j0 + jj;
      // groups of UNR rows, folded every kRB / UNR groups outside the inner
      // loop (a fold test per group is if-converted into masked FP64 work on
      // every group).  The branch-free df_step measured slower here.
      while (j + (UNR - 1) * G < j1) {
        for (int g = 0; g < kRB / UNR && j + (UNR - 1) * G < j1; g++, j += UNR * G, p += UNR * st) {
          typename E::C r[UNR][1];
#pragma unroll
          for (int q = 0; q < UNR; q++) E::template load<1>(p + q * st, r[q]);
#pragma unroll
          for (int q = 0; q < UNR; q++) acc.emul1(0, r[q][0], x + j + q * G, ldxs(a.xs + j + q * G));
        }
        acc.fold();
      }
      for (; j < j1; j += G, p += st) {
        typename E::C r[1];
        E::template load<1>(p, r);
        acc.emul1(0, r[0], x + j, ldxs(a.xs + j));
      }
    }
    acc.fold();
    tot = active ? acc.result(0) : 0.0;
  } else {
    AccF32<1> acc;
    acc.init();
    int blk = 0;  // (the FP32 fold is cheap enough to test per group)
    if (active) {
      int64_t j = j0 + jj;
      for (; j + (UNR - 1) * G < j1; j += UNR * G, p += UNR * st) {
        float r[UNR][1];
#pragma unroll
        for (int q = 0; q < UNR; q++) E::template load<1>(p + q * st, r[q]);
#pragma unroll
        for (int q = 0; q < UNR; q++) acc.a[0] = __fmaf_rn(r[q][0], xval(a, j + q * G), acc.a[0]);
        if (++blk == kRB / UNR) {
          acc.fold();
          blk = 0;
        }
      }
      for (; j < j1; j += G, p += st) {
        float r[1];
        E::template load<1>(p, r);
        acc.a[0] = __fmaf_rn(r[0], xval(a, j), acc.a[0]);
      }
    }
    acc.fold();
    tot = active ? acc.result(0) : 0.0f;
  }
  // Sum the G lanes that share l: lane jj*v + l, jj = 0..G-1.
  for (int k = 1; k < G; k <<= 1) {
    V other = __shfl_down_sync(0xFFFFFFFFu, tot, k * (int)a.v);
    if (jj + k < G) tot += other;
  }
  if (jj == 0) {
    if constexpr (kF64Acc<DT>)
      emit(a, blockIdx.y, slab * a.v + l, tot);
    else
      emit(a, blockIdx.y, slab * a.v + l, __fmul_rn(tot, out_scale(a, slab)));
  }
}

// ------------------------------------------------------------------ TILE --

// One block contracts R whole slabs (R*S contiguous elements, S = n_k*v)
// staged in shared memory, with x staged beside them.  Thread t < R*v owns
// output (r, l) = (t / v, t % v).  For v == 1 and even n_k each thread starts
// its row at a rotated position so the warp's shared-memory reads spread
// over the banks.
template <tvc_dtype DT>
__global__ void __launch_bounds__(kThreads) tvc_tile_kernel(const TvcArgs<DT> a, int R, int vec16) {
  if (skip(a.done)) return;
  using E = Elem<DT>;
  using T = typename E::T;
  extern __shared__ __align__(128) unsigned char smraw[];
  const int64_t S = a.nk * a.v;
  const int nk = (int)a.nk, v = (int)a.v;
  const int64_t i0 = (int64_t)blockIdx.x * R;
  const int Reff = (int)min((int64_t)R, a.u - i0);
  T* sm = reinterpret_cast<T*>(smraw);
  const size_t tile_bytes = ((size_t)R * S * sizeof(T) + 15) / 16 * 16;
  const int t = threadIdx.x;
  // Stage x.
  if constexpr (kF64Acc<DT>) {
    XSplit* smx = reinterpret_cast<XSplit*>(smraw + tile_bytes);
    for (int j = t; j < nk; j += kThreads) smx[j] = ldxs(a.xs + j);
  } else {
    float* smx = reinterpret_cast<float*>(smraw + tile_bytes);
    for (int j = t; j < nk; j += kThreads) smx[j] = xval(a, j);
  }
  // Stage the tile: R*S contiguous elements.
  const T* src = a.A + i0 * S;
  const int64_t total = (int64_t)Reff * S;
  const int64_t bytes = total * (int64_t)sizeof(T);
  int64_t done = 0;
  if (vec16) {
    const int64_t n16 = bytes / 16;
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(sm);
    int64_t q = t;
    for (; q + 3 * kThreads < n16; q += 4 * kThreads) {
      uint4 r0 = __ldcs(s4 + q), r1 = __ldcs(s4 + q + kThreads), r2 = __ldcs(s4 + q + 2 * kThreads),
            r3 = __ldcs(s4 + q + 3 * kThreads);
      d4[q] = r0;
      d4[q + kThreads] = r1;
      d4[q + 2 * kThreads] = r2;
      d4[q + 3 * kThreads] = r3;
    }
    for (; q < n16; q += kThreads) d4[q] = __ldcs(s4 + q);
    done = n16 * 16 / (int64_t)sizeof(T);
  }
  for (int64_t e = done + t; e < total; e += kThreads)
    reinterpret_cast<RawVec<sizeof(T)>*>(sm)[e] = ld_stream<sizeof(T)>(src + e);
  __syncthreads();
  if (t >= Reff * v) return;
  const int r = t / v, l = t - (t / v) * v;
  const int rot = (v == 1 && (nk & 1) == 0) ? r % nk : 0;
  const T* row = sm + (int64_t)r * S + l;
  int jt = rot;
  int blk = 0;
  if constexpr (kF64Acc<DT>) {
    const double* x = static_cast<const double*>(a.x);
    const XSplit* smx = reinterpret_cast<const XSplit*>(smraw + tile_bytes);
    AccF64<1> acc;
    acc.init();
    for (int cb = 0; cb < nk; cb += kRB) {  // fold outside the inner loop
      const int ce = min(nk, cb + kRB);
      for (int c = cb; c < ce; c++) {
        acc.emul1(0, row[(int64_t)jt * v], x + jt, smx[jt]);
        if (++jt == nk) jt = 0;
      }
      acc.fold();
    }
    emit(a, 0, (i0 + r) * a.v + l, acc.result(0));
  } else {
    const float* smx = reinterpret_cast<const float*>(smraw + tile_bytes);
    AccF32<1> acc;
    acc.init();
    for (int c = 0; c < nk; c++) {
      float val[1];
      E::template load<1, true>(row + (int64_t)jt * v, val);
      acc.a[0] = __fmaf_rn(val[0], smx[jt], acc.a[0]);
      if (++jt == nk) jt = 0;
      if (++blk == kRB) {
        acc.fold();
        blk = 0;
      }
    }
    acc.fold();
    emit(a, 0, (i0 + r) * a.v + l, __fmul_rn(acc.result(0), out_scale(a, i0 + r)));
  }
}

// Small slabs, persistent and double-buffered: block b contracts tiles
// b, b + grid, ... of R whole slabs (R*S contiguous elements).  Each tile is
// fetched with 16-byte cp.async chunks from the 16-byte boundary at or below
// its first byte (A is 16-byte aligned, so every chunk starts inside A); the
// one chunk that would run past the end of A is read element by element.
// The next tile is in flight while the current one is contracted: thread
// t < R*v owns output (r, l) = (t / v, t % v) and reads its n_k entries from
// shared memory with stride v.  One tile per block with plain loads (the
// kernel above) serialised a DRAM round trip per load step whenever R*S*s_A
// was not a multiple of 16.
template <tvc_dtype DT>
__global__ void __launch_bounds__(kThreads) tvc_tile_async_kernel(const TvcArgs<DT> a, int R, int64_t ntiles,
                                                                  int tile_cap) {
  if (skip(a.done)) return;
  using E = Elem<DT>;
  using T = typename E::T;
  constexpr int es = (int)sizeof(T);
  extern __shared__ __align__(128) unsigned char smraw[];
  const int64_t S = a.nk * a.v;
  const int nk = (int)a.nk, v = (int)a.v;
  const int t = threadIdx.x;
  if ((int64_t)blockIdx.x >= ntiles) return;
  const int x_bytes = ((nk * (kF64Acc<DT> ? (int)sizeof(XSplit) : 4)) + 15) / 16 * 16;
  unsigned char* const buf0 = smraw + x_bytes;  // buffer k at buf0 + k * tile_cap
  __shared__ int x_out;  // FP64: some x_j outside the exact window
  if constexpr (kF64Acc<DT>) {
    XSplit* smx = reinterpret_cast<XSplit*>(smraw);
    if (t == 0) x_out = 0;
    __syncthreads();
    int bad = 0;
    for (int j = t; j < nk; j += kThreads) {
      smx[j] = ldxs(a.xs + j);
      bad |= (smx[j].xh != smx[j].xh);
    }
    if (bad) atomicOr(&x_out, 1);
  } else {
    float* smx = reinterpret_cast<float*>(smraw);
    for (int j = t; j < nk; j += kThreads) smx[j] = xval(a, j);
  }
  const char* A0 = reinterpret_cast<const char*>(a.A);
  const char* Aend = A0 + a.u * S * es;
  // Queues tile `tile` into `dst`; returns the byte offset of its first element.
  auto issue = [&](int64_t tile, unsigned char* dst) -> int {
    const int64_t i0 = tile * R;
    const int64_t reff = min((int64_t)R, a.u - i0);
    const char* gs = A0 + i0 * S * es;
    const char* ge = gs + reff * S * es;
    const char* c0 = A0 + ((gs - A0) & ~(int64_t)15);
    const int64_t nch = (ge - c0 + 15) / 16;
    for (int64_t q = t; q < nch; q += kThreads) {
      const char* src = c0 + 16 * q;
      if (src + 16 <= Aend) {
        cp_async16(dst + 16 * q, src);
      } else {
        for (const char* e = src; e < Aend; e += es)
          *reinterpret_cast<RawVec<es>*>(dst + 16 * q + (e - src)) = ld_plain<es>(e);
      }
    }
    return (int)(gs - c0);
  };
  int head0 = issue(blockIdx.x, buf0), head1 = 0;  // first-element offsets in buffers 0 and 1
  cp_async_commit();
  int k = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, k ^= 1) {
    const int64_t nxt = tile + gridDim.x;
    if (nxt < ntiles) {
      if (k == 0) head1 = issue(nxt, buf0 + tile_cap);
      else head0 = issue(nxt, buf0);
    }
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const int64_t i0 = tile * R;
    const int reff = (int)min((int64_t)R, a.u - i0);
    if (t < reff * v) {
      const int r = t / v, l = t - (t / v) * v;
      const T* row = reinterpret_cast<const T*>(buf0 + k * tile_cap + (k ? head1 : head0)) + (int64_t)r * S + l;
      if constexpr (kF64Acc<DT>) {
        const double* x = static_cast<const double*>(a.x);
        const XSplit* smx = reinterpret_cast<const XSplit*>(smraw);
        // Branch-free float-float products with the window bits ORed
        // alongside; an output that met an element (or x) outside the exact
        // window is recomputed with DFMA.  Blocks of kRB products are folded
        // outside the inner loop: a fold test inside it is if-converted, and
        // its FP64 instructions then issue (masked off) for every element.
        double d = 0.0;
        uint32_t bad = (uint32_t)x_out;
        for (int jb = 0; jb < nk; jb += kRB) {
          const int je = min(nk, jb + kRB);
          float sf = 0.0f, cf = 0.0f;
          for (int j = jb; j < je; j++) {
            const auto aj = row[j * v];  // binary64, or binary32 promoted in the product
            bad |= df_out_of_window(aj);
            df_mac_fast(sf, cf, aj, smx[j]);
          }
          d += (double)sf;
          d += (double)cf;
        }
        if (bad) {
          d = 0.0;
          for (int j = 0; j < nk; j++) d = fma((double)row[j * v], x[j], d);
        }
        emit(a, 0, (i0 + r) * a.v + l, d);
      } else {
        const float* smx = reinterpret_cast<const float*>(smraw);
        AccF32<1> acc;
        acc.init();
        for (int jb = 0; jb < nk; jb += kRB) {
          const int je = min(nk, jb + kRB);
          for (int j = jb; j < je; j++) {
            float val[1];
            E::template load<1, true>(row + j * v, val);
            acc.a[0] = __fmaf_rn(val[0], smx[j], acc.a[0]);
          }
          acc.fold();
        }
        emit(a, 0, (i0 + r) * a.v + l, __fmul_rn(acc.result(0), out_scale(a, i0 + r)));
      }
    }
    __syncthreads();  // buf[k] is refilled two tiles on
  }
  cp_async_wait<0>();
}

// Large slabs (1 < v < 32) of the narrow types and FP32: one block per slab (and
// split of n_k) streams its rows in tiles of about 8 KB, copied from the
// 16-byte boundary below the tile with cp.async into two shared-memory
// buffers (the next tile in flight while the current one is used); thread
// (ph, c) of P = floor(256 / (v / W)) phases sums the rows j = ph (mod P)
// of its W columns c*W .. c*W + W-1 from shared memory (one load and one x
// entry per W elements), and the P partial sums of each column are added
// in phase order at the end.  The per-warp slab kernel reads 1- or 2-byte
// elements straight from global memory; here every global access is a
// 16-byte piece.
constexpr int kSlabTile = 8192;  // bytes of A per tile

template <tvc_dtype DT, int W>
__global__ void __launch_bounds__(kThreads) tvc_slab_async_kernel(const TvcArgs<DT> a) {
  if (skip(a.done)) return;
  using E = Elem<DT>;
  using T = typename E::T;
  constexpr int es = (int)sizeof(T);
  __shared__ __align__(16) unsigned char buf[2][kSlabTile + 32];
  __shared__ float red[kThreads * W];
  const int v = (int)a.v;
  const int C = v / W;       // threads per row, W consecutive columns each
  const int P = kThreads / C;
  const int t = threadIdx.x;
  const int ph = t / C, l = (t - (t / C) * C) * W;
  const bool act = ph < P;
  const int64_t i = blockIdx.x;
  const int64_t j0 = (int64_t)blockIdx.y * a.chunk;
  const int64_t j1 = min(a.nk, j0 + a.chunk);
  const int J = kSlabTile / (v * es);  // rows per tile
  const char* A0 = reinterpret_cast<const char*>(a.A);
  const char* Aend = A0 + a.u * a.nk * a.v * es;
  // Queues rows [jt, jt + n) of slab i into dst; returns the first element's byte offset.
  auto issue = [&](int64_t jt, int n, unsigned char* dst) -> int {
    const char* gs = A0 + ((i * a.nk + jt) * a.v) * es;
    const char* ge = gs + (int64_t)n * v * es;
    const char* c0 = A0 + ((gs - A0) & ~(int64_t)15);
    const int nch = (int)((ge - c0 + 15) / 16);
    for (int q = t; q < nch; q += kThreads) {
      const char* src = c0 + 16 * q;
      if (src + 16 <= Aend) {
        cp_async16(dst + 16 * q, src);
      } else {
        for (const char* e = src; e < Aend; e += es)
          *reinterpret_cast<RawVec<es>*>(dst + 16 * q + (e - src)) = ld_plain<es>(e);
      }
    }
    return (int)(gs - c0);
  };
  AccF32<W> acc;
  acc.init();
  int head[2] = {0, 0};
  head[0] = issue(j0, (int)min((int64_t)J, j1 - j0), buf[0]);
  cp_async_commit();
  int k = 0, blk = 0;
  for (int64_t jt = j0; jt < j1; jt += J, k ^= 1) {
    const int n = (int)min((int64_t)J, j1 - jt);
    if (jt + J < j1) head[k ^ 1] = issue(jt + J, (int)min((int64_t)J, j1 - jt - J), buf[k ^ 1]);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    if (act) {
      const T* tile = reinterpret_cast<const T*>(buf[k] + head[k]);
      for (int jl = ph; jl < n; jl += P) {
        float val[W];
        E::template load<W, true>(tile + jl * v + l, val);  // W * es bytes, aligned (see the planner)
        acc.mac(val, xval(a, jt + jl));
        if (++blk == kRB) {
          acc.fold();
          blk = 0;
        }
      }
    }
    __syncthreads();  // buf[k] is refilled two tiles on
  }
  cp_async_wait<0>();
  acc.fold();
#pragma unroll
  for (int e = 0; e < W; e++) red[ph * v + l + e] = act ? acc.result(e) : 0.0f;  // (ph, column)
  __syncthreads();
  if (t < v) {
    float sum = red[t];
    for (int q = 1; q < P; q++) sum = __fadd_rn(sum, red[q * v + t]);  // phases in order
    emit(a, blockIdx.y, i * a.v + t, __fmul_rn(sum, out_scale(a, i)));
  }
}

// -------------------------------------------------------- helper kernels --

// xs[j] = split pieces of x[j]; with xs1 (nullable) also xs1[j + 1] = xs[j]
// and zero pieces at xs1[0] and xs1[n + 1].
__global__ void tvc_split_x_kernel(const double* __restrict__ x, XSplit* __restrict__ xs, XSplit* __restrict__ xs1,
                                   int64_t n, const int* done) {
  if (skip(done)) return;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const XSplit t = split_x(x[j]);
    xs[j] = t;
    if (xs1) xs1[j + 1] = t;
  }
  if (xs1 && blockIdx.x == 0 && threadIdx.x == 0) {
    xs1[0] = XSplit{0.0f, 0.0f};
    xs1[n + 1] = XSplit{0.0f, 0.0f};
  }
}

// y[o] = alpha * sum_s partial[s][o] + beta * y[o], s ascending (deterministic).
template <class V>
__global__ void tvc_reduce_kernel(const V* __restrict__ partial, V* __restrict__ y, int64_t uv, int64_t splits,
                                  double alpha, double beta, const int* done) {
  if (skip(done)) return;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < uv; o += (int64_t)gridDim.x * blockDim.x) {
    V r;
    if constexpr (sizeof(V) == 8) {
      double s = 0.0;
      for (int64_t k = 0; k < splits; k++) s += partial[k * uv + o];
      r = alpha * s;
      if (beta != 0.0) r += beta * y[o];
    } else {
      KahanF32 s;
      for (int64_t k = 0; k < splits; k++) s.add(partial[k * uv + o]);
      r = (float)alpha * s.value();
      if (beta != 0.0) r += (float)beta * y[o];
    }
    y[o] = r;
  }
}

// ------------------------------------------------------------------ plan --

enum Kind {
  K_COLS = 0,
  K_ROWS = 1,
  K_SLAB = 2,
  K_TILE = 3,
  K_ROWS_SHORT = 4,
  K_ROWS_TMA = 5,
  K_ROWS_F64S = 6,
  K_ROWS_MULTI = 7,
  K_TILE_ASYNC = 8,
  K_SLAB_ASYNC = 9,
  K_F64_TILE = 10,
  K_SLAB_TILE = 11
};

struct Plan {
  Kind kind = K_COLS;
  int vec = 1;
  int64_t splits = 1, chunk = 0;
  int R = 0, vec16 = 0, g = 0, G = 0, nst = 0, RW = 0, S = 0, dq = 0, rb = 0, unr = 0;
  int64_t ntiles = 0;
  uint32_t tile_bytes = 0;
  size_t smem = 0;
  dim3 grid;
  F64TileParams ft{};
  SlabTileParams st{};
  int xs_shift = 0;  // FP64 rows of odd length with 16-byte pairs: the shifted split x too
  size_t ws_xs = 0, ws_partial = 0, ws_total = 0;
};

// Opts a kernel in to `bytes` of dynamic shared memory, once per kernel and
// device (the attribute is per device function).
static void opt_in_smem(const void* kern, int bytes) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (done.insert({dev, kern}).second) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    // prefer the largest shared-memory carveout so that two blocks fit
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  }
}

// Measured defaults of the planner (one choice per case; no run-time
// switches).  Staged (TMA) rows kernel: 4 steps per lane (fewer registers
// than 8).  FP64 rows with 8-byte loads (odd n_k) of up to 4096 elements go
// to the slots kernel with G = 32 (below that the per-row FP64 epilogue of
// one row per warp occupies the FP64 pipe; 979-element rows 4.0 -> 5.3
// TB/s).
constexpr int kStagedSteps = 4;
constexpr int64_t kF64SlotsMaxNk = 4096;

// Rows in flight per lane of the slab kernel: 8 for FP64/FP32, 16 for the
// narrow types (measured at v = 3 .. 20).
static int slab_unroll(tvc_dtype dt) { return (dt == TVC_BF16 || dt == TVC_E4M3 || dt == TVC_F16) ? 16 : 8; }

// Rows per warp (2, 4 or 8) and unrolled steps (1 or 2) of the narrow
// long-row kernel, per storage type as measured on rows of 16384 to 1048576
// elements: E4M3 8 x 1 (x traffic 0.5x that of A, 128 registers), BF16 2 x 2,
// FP32 4 x 2.
static int rows_multi_rb(tvc_dtype dt) {
  return dt == TVC_E4M3 ? 8 : ((dt == TVC_BF16 || dt == TVC_F16) ? 2 : 4);
}
static int rows_multi_unr(tvc_dtype dt) { return dt == TVC_E4M3 ? 1 : 2; }

// Largest vector width (elements per load) the alignment and v allow.
static int pick_vec(tvc_dtype dt, int64_t stride_elems, const void* A, int max_vec = 16) {
  const int es = (int)elem_size(dt);
  const int cands[3] = {16 / es, 4 / es > 1 ? 4 / es : 1, 1};
  for (int c : cands) {
    if (c <= 1) return 1;
    if (c > max_vec) continue;
    if (stride_elems % c == 0 && aligned(A, (size_t)c * es)) return c;
  }
  return 1;
}

static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

static Plan make_plan_impl(const Shape& s, tvc_dtype dt, const void* A, bool allow_staged);
static Plan make_plan_unstaged(const Shape& s, tvc_dtype dt, const void* A) {
  return make_plan_impl(s, dt, A, false);
}
static Plan make_plan(const Shape& s, tvc_dtype dt, const void* A) { return make_plan_impl(s, dt, A, true); }

// Persistent double-buffered tiles of whole slabs, one thread per output
// (the small-slab kernel): R slabs of S = n_k * v elements per tile.
static void plan_tile_async(Plan& p, const Shape& s, size_t es, bool f64acc, int sms) {
  const int64_t S = s.nk * s.v;
  p.kind = K_TILE_ASYNC;
  int64_t R = std::min<int64_t>(kThreads / s.v, (int64_t)(48 * 1024) / (int64_t)(S * es));
  R = std::max<int64_t>(1, std::min<int64_t>(R, s.u));
  p.R = (int)R;
  p.ntiles = ceil_div(s.u, R);
  p.vec16 = (int)(align_up((size_t)R * S * es, 16) + 32);  // tile capacity in bytes
  const size_t x_bytes = align_up((size_t)s.nk * (f64acc ? sizeof(XSplit) : 4), 16);
  p.smem = x_bytes + 2 * (size_t)p.vec16;
  const int bps = (int)std::max<size_t>(1, std::min<size_t>(8, (size_t)(220 * 1024) / p.smem));
  p.splits = 1;
  p.chunk = s.nk;
  p.grid = dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(p.ntiles, (int64_t)sms * bps)), 1);
}

// FP64-arithmetic rows (v = 1) that go to the small-slab kernel, one thread
// per row from shared-memory tiles: 9 .. 27 elements, except 16, 20 and 24,
// where the grouped-row kernel's 16-byte passes come out even.  Measured on
// 1 GB tensors (n_k = 2 .. 31): 1.1-2.8x faster in that range (10 elements:
// 35% -> 65% of the copy peak, 12: 28% -> 66%, 19: 52% -> 64%), slower at
// 16, 20, 24 (81% -> 33%, 80% -> 65%, 76% -> 49%) and for rows of <= 8.
static bool f64_rows_by_tiles(int64_t nk) { return nk >= 9 && nk <= 27 && !(nk % 4 == 0 && nk >= 16); }

// FP64 small slabs and short rows through the copy-engine tile kernel
// (tvc_f64tile.cu).  G, the lanes per output, is the smallest power of two
// that keeps a lane at <= 32 steps per output (the error model allows 64
// products per compensated sum) and fits two stages of at least one pass of
// outputs into a block's share of shared memory (two blocks per SM): with
// fewer than ~16 steps per lane the per-output work (group reduction,
// slots) measured 10-20% slower.  Tiles are up to 54 KB of whole passes
// (v = 1) or whole slabs (v > 1: the count that leaves the fewest idle
// lanes, and G raised while that leaves more than 15% of them idle).  Rows whose length is a multiple of 4 (8 or more) are copied as
// 2-D boxes with a padded row of n_k + 2 elements (their plain starts fall
// on 8 or fewer of the 16 shared-memory bank pairs); they need
// G | n_k / 2 (no step reads the zero columns) and n_k + 2 <= 256 (the box
// limit).  Rows of 4 measured faster in the grouped-row kernel.
constexpr int64_t kFtTileMax = 54 * 1024;     // bytes of one tile
constexpr int64_t kFtBlockSmem = 111 * 1024;  // shared memory of one block: two blocks per SM
constexpr int kFtQMax = 32;                   // steps per lane and output

static bool plan_f64_tile_g(Plan& p, const Shape& s, int sms, double min_util);
static bool plan_f64_tile(Plan& p, const Shape& s, int sms) {
  // slabs: the smallest G whose tiles keep >= 85% of the lanes busy, else
  // the smallest G at all
  return plan_f64_tile_g(p, s, sms, s.v > 1 ? 0.85 : 0.0) || (s.v > 1 && plan_f64_tile_g(p, s, sms, 0.0));
}

static bool plan_f64_tile_g(Plan& p, const Shape& s, int sms, double min_util) {
  if (s.v >= 32 || s.nk < 2 || s.nk > 32 * kFtQMax) return false;
  const bool pad = s.v == 1 && s.nk % 4 == 0;
  if (pad && (s.nk < 8 || s.nk + 2 > 256 || s.u >= ((int64_t)1 << 30) || encode_tiled() == nullptr)) return false;
  const int64_t S = s.nk * s.v;
  const int64_t srow = pad ? s.nk + 2 : S;
  for (int G = 1; G <= 32; G *= 2) {
    if (pad && s.nk % (2 * G) != 0) break;
    const int64_t Q = ceil_div(s.nk, G);
    if (Q > kFtQMax) continue;
    const int64_t OPP = 256 / G;
    int64_t R = 0;
    if (s.v == 1) {
      if (OPP * srow * 8 > kFtTileMax) continue;
      R = OPP * (kFtTileMax / (OPP * srow * 8));
      if (pad && R > 256) R = R / 256 * 256;  // whole boxes of 256 rows
    } else {
      const int64_t rmax = kFtTileMax / (S * 8);
      double best = -1.0;
      for (int64_t r = 1; r <= rmax; r++) {
        if ((r * S) % 2 != 0) continue;
        const int64_t outs = r * s.v, passes = ceil_div(outs, OPP);
        const double util = (double)outs / (double)(passes * OPP);
        if (util >= best) {
          best = util;
          R = r;
        }
      }
      if (R == 0) return false;  // slabs too large for a tile
      if (best < min_util) continue;
    }
    // one tile (then the last) when u is smaller; padded rows keep whole
    // boxes (rows past u arrive as zeros)
    if (!pad) R = std::min<int64_t>(R, s.u);
    const int npairs = (int)ceil_div(Q, 2);
    const int64_t over = pad ? 0 : (2 * (int64_t)npairs * G - s.nk) * s.v;  // padded steps past a tile's end
    const int64_t stride = (int64_t)align_up((size_t)(R * srow * 8 + over * 8), 128) + 128;
    const int64_t fixed = (int64_t)G * npairs * 16 + 16 * 8;  // x pieces and barriers
    const int NS = (int)std::min<int64_t>(8, (kFtBlockSmem - fixed) / stride);
    if (NS < 2) continue;
    p.kind = K_F64_TILE;
    p.ft.R = (int)R;
    p.ft.G = G;
    p.ft.NS = NS;
    p.ft.npairs = npairs;
    p.ft.ntiles = ceil_div(s.u, R);
    p.ft.stage_bytes = (uint32_t)stride;
    p.ft.srow = (int)srow;
    p.ft.box_rows = pad ? (int)std::min<int64_t>(R, 256) : 0;
    p.ft.w16 = (G == 1 && s.v == 1 && srow % 2 == 0) ? 1 : 0;
    p.smem = f64tile_smem_bytes(p.ft);
    p.splits = 1;
    p.chunk = s.nk;
    p.grid = dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(p.ft.ntiles, (int64_t)sms * 2)), 1);
    return true;
  }
  return false;
}

// Large slabs whose rows are whole 16-byte pieces (v * element size = 16,
// 32, 64 or 128 bytes: BF16 / F16 v = 8, 16; E4M3 v = 16; FP32 v = 4, 8,
// 16), FP32 accumulators: the copy-engine slab kernel (tvc_slabtile.cu).
// Tiles of up to 48 KB of rows (at most 64 rows per thread; two stages in a
// block's 111 KB: measured against 32 KB x 3, 24 KB x 4 and 16 KB x 6 on
// 4096x4096x16 and 8192x4096x16, BF16 5.35 -> 5.59 and 5.80 -> 5.99 TB/s),
// the rows of a slab split when the slabs alone give fewer than 8 work
// items per SM.
constexpr int64_t kStTileMax = 48 * 1024;
constexpr int64_t kStBlockSmem = 111 * 1024;

static bool plan_slab_tile(Plan& p, const Shape& s, tvc_dtype dt, int sms) {
  const int64_t rb = s.v * (int64_t)elem_size(dt);
  if (s.v < 2 || s.v >= 32 || rb % 16 != 0 || s.nk < 256) return false;
  const int CPR = (int)(rb / 16);
  if (CPR != 1 && CPR != 2 && CPR != 4 && CPR != 8) return false;
  const int64_t P = 256 / CPR;
  int64_t TR = std::min<int64_t>(kStTileMax / rb, 64 * P);
  const int64_t target = (int64_t)sms * 8;
  int64_t splits = 1;
  if (s.u < target) splits = std::min(ceil_div(target, s.u), std::max<int64_t>(1, s.nk / TR));
  p.chunk = ceil_div(s.nk, splits);
  p.splits = ceil_div(s.nk, p.chunk);
  TR = std::min<int64_t>(TR, p.chunk);
  const int64_t stride = (int64_t)align_up((size_t)(TR * rb), 128);
  const int64_t part = (int64_t)align_up((size_t)8 * s.v * 4, 16);
  const int NS = (int)std::min<int64_t>(8, (kStBlockSmem - part - 128) / stride);
  if (NS < 2) return false;
  p.kind = K_SLAB_TILE;
  p.st.TR = (int)TR;
  p.st.NS = NS;
  p.st.CPR = CPR;
  p.st.splits = p.splits;
  p.st.chunk = p.chunk;
  p.st.nitems = s.u * p.splits;
  p.st.stage_bytes = (uint32_t)stride;
  p.st.part_bytes = (uint32_t)part;
  p.smem = slabtile_smem_bytes(p.st);
  p.grid = dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(p.st.nitems, (int64_t)sms * 2)), 1);
  return true;
}

static Plan make_plan_impl(const Shape& s, tvc_dtype dt, const void* A, bool allow_staged) {
  Plan p;
  const bool f64acc = (dt == TVC_F64 || dt == TVC_F32D);  // FP64 arithmetic (float-float kernels)
  const int sms = device_sms();
  const int64_t target_threads = (int64_t)sms * 2048;
  const int64_t S = s.nk * s.v;
  const size_t es = elem_size(dt);
  if (s.v >= 32) {
    p.kind = K_COLS;
    p.vec = pick_vec(dt, s.v, A);
    const int64_t threads = ceil_div(s.uv, p.vec);
    int64_t splits = 1;
    if (threads < target_threads) splits = std::min(ceil_div(target_threads, threads), std::max<int64_t>(1, s.nk / 64));
    p.chunk = ceil_div(ceil_div(s.nk, splits), 8) * 8;
    p.splits = ceil_div(s.nk, p.chunk);
    p.grid = dim3((unsigned)ceil_div(threads, kThreads), (unsigned)p.splits);
  } else if (dt == TVC_F64 && aligned(A, 16) && s.v < 32 && plan_f64_tile(p, s, sms)) {
    // FP64 small slabs and short rows: the copy-engine tile kernel.
  } else if (s.v == 1 && !f64acc && allow_staged && aligned(A, 16) &&
             s.nk <= 8 * 32 * (int64_t)pick_vec(dt, s.nk, A, 4) && s.u >= 8) {
    // Staged short rows: tiles of R = 8*RW whole rows through shared memory.
    p.kind = K_ROWS_TMA;
    p.vec = pick_vec(dt, s.nk, A, 4);
    int G = 1;
    while (G < 32 && (int64_t)G * p.vec * kStagedSteps < s.nk) G <<= 1;
    p.G = G;
    p.nst = (int)ceil_div(s.nk, (int64_t)G * p.vec);
    p.dq = 0;
    const int gpw = kWarp / G;
    const int64_t row_bytes = s.nk * (int64_t)es;
    int RW = gpw;  // at least one row per group
    while (RW * 2 <= 32 && (int64_t)kTmaConsumerWarps * RW * 2 * row_bytes <= 24 * 1024) RW *= 2;
    // tiles must keep 16-byte alignment of every tile start and stage buffer
    while (((int64_t)kTmaConsumerWarps * RW * row_bytes) % 16 != 0 && RW < 64) RW *= 2;
    p.RW = RW;
    if (((int64_t)kTmaConsumerWarps * RW * row_bytes) % 16 != 0) {
      // cannot happen for 8 warps and RW a power of two >= 2 (8*2*es*n_k is a
      // multiple of 16); kept as a guard: fall back to the register kernels.
      return make_plan_unstaged(s, dt, A);
    }
    p.R = kTmaConsumerWarps * RW;
    p.tile_bytes = (uint32_t)(p.R * row_bytes);
    p.S = (int)std::max<int64_t>(2, std::min<int64_t>(6, (int64_t)(96 * 1024) / p.tile_bytes));
    p.ntiles = ceil_div(s.u, p.R);
    p.smem = (size_t)p.S * p.tile_bytes + (size_t)kTmaConsumerWarps * RW * (sizeof(float2) + sizeof(double)) +
             2 * (size_t)p.S * sizeof(uint64_t);
    p.splits = 1;
    p.chunk = s.nk;
    p.grid = dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(p.ntiles, (int64_t)sms * 2)), 1);
  } else if (s.v == 1 && !f64acc && s.nk <= 8 * 32 * (int64_t)pick_vec(dt, s.nk, A, 4)) {
    // (FP64 rows, short or long, measured fastest with the grouped-row
    // kernel below; the staged kernel serves the narrow types.)
    // Short rows: the smallest group whose 4 steps cover the row (8 steps
    // at G = 32); each group takes several rows per iteration (see the
    // kernel) so that enough loads are in flight.
    p.kind = K_ROWS_SHORT;
    p.vec = pick_vec(dt, s.nk, A, 4);
    int G = 1;
    while (G < 32 && (int64_t)G * p.vec * 4 < s.nk) G <<= 1;
    p.G = G;
    const int64_t nst = ceil_div(s.nk, (int64_t)G * p.vec);
    p.nst = nst <= 2 ? 2 : (nst <= 4 ? 4 : 8);
    const int B = std::max(1, std::min(4, 32 / (p.nst * p.vec)));  // as in the kernel
    const int64_t rows_per_block = (int64_t)kWarpsPerBlock * (kWarp / G) * B;
    const int64_t blocks = std::min<int64_t>(ceil_div(s.u, rows_per_block), (int64_t)sms * 4);
    p.splits = 1;
    p.chunk = s.nk;
    p.grid = dim3((unsigned)std::max<int64_t>(1, blocks), 1);
  } else if (s.v == 1 && !f64acc && pick_vec(dt, s.nk, A) * (int)es == 16) {
    // Long rows of the narrow types: RB rows per warp share each x piece.
    p.kind = K_ROWS_MULTI;
    p.vec = pick_vec(dt, s.nk, A);
    p.rb = rows_multi_rb(dt);
    p.unr = rows_multi_unr(dt);
    const int64_t step = (int64_t)kWarp * p.vec;
    const int64_t warps = ceil_div(s.u, p.rb);
    const int64_t target_warps = (int64_t)sms * 48;
    int64_t splits = 1;
    if (warps < target_warps) splits = std::min(ceil_div(target_warps, warps), std::max<int64_t>(1, s.nk / (4 * step)));
    p.chunk = ceil_div(ceil_div(s.nk, splits), step) * step;
    p.splits = ceil_div(s.nk, p.chunk);
    p.grid = dim3((unsigned)ceil_div(warps, kWarpsPerBlock), (unsigned)p.splits);
  } else if (s.v == 1 && f64acc && aligned(A, 16) && f64_rows_by_tiles(s.nk)) {
    plan_tile_async(p, s, es, f64acc, sms);
  } else if (s.v == 1) {
    p.kind = K_ROWS;
    p.vec = pick_vec(dt, s.nk, A);
    if (dt == TVC_F64 && p.vec == 1 && s.nk % 2 == 1 && s.nk >= 1024 && aligned(A, 16)) {
      // FP64 rows of odd length: 16-byte pairs from the first 16-byte
      // boundary of each row segment, the pieces of x from a copy shifted by
      // one entry where that boundary falls on an odd element (measured on
      // rows of 1025 .. 100001: 2-12% faster than 8-byte loads, 2.4x at
      // 4095; below 1024 the slots kernel stays faster).
      p.vec = 2;
      p.xs_shift = 1;
    }
    // Lanes per row: the largest power of two <= 32 that still gives every
    // lane at least four loads of its row (at least 2 lanes; FP64 short rows
    // go down to 1 lane, so that rows of 8 .. 15 elements fill one unrolled
    // pass of the slots kernel).
    int G = 32;
    const int gmin = f64acc ? 1 : 2;
    while (G > gmin && (int64_t)G * p.vec * 4 > s.nk) G >>= 1;
    p.G = G;
    const int64_t group = 4 * (int64_t)G * p.vec;  // one unrolled step of a group
    int64_t rows_per_block = (int64_t)kWarpsPerBlock * (kWarp / G);
    if (f64acc && (G < 32 || (p.vec == 1 && s.nk <= kF64SlotsMaxNk))) {
      p.kind = K_ROWS_F64S;  // 32 rows per warp, results converted in slots
      rows_per_block = (int64_t)kWarpsPerBlock * kWarp;
    }
    const int64_t target_groups = (int64_t)sms * 64 * (kWarp / G);
    int64_t splits = 1;
    if (s.u < target_groups) splits = std::min(ceil_div(target_groups, s.u), std::max<int64_t>(1, s.nk / (8 * group)));
    // FP64 rows whose split x (8 bytes an entry) outgrows L1, enough rows to
    // fill the GPU: segments of about 4096 entries, so that the blocks
    // working on one segment (the grid runs rows fastest) share its pieces
    // of x in L1 (30623-element rows: 77% -> 82% of the copy peak); not when
    // the segments' partial sums would pass 16 MB of workspace.
    if (f64acc && splits == 1 && s.nk * (int64_t)sizeof(XSplit) > 160 * 1024 &&
        s.u * ceil_div(s.nk, 4096) * (int64_t)sizeof(double) <= 16 * 1024 * 1024)
      splits = ceil_div(s.nk, 4096);
    p.chunk = ceil_div(ceil_div(s.nk, splits), group) * group;
    p.splits = ceil_div(s.nk, p.chunk);
    p.grid = dim3((unsigned)ceil_div(s.u, rows_per_block), (unsigned)p.splits);
  } else if (!f64acc && aligned(A, 16) && plan_slab_tile(p, s, dt, sms)) {
    // large slabs of whole 16-byte rows: the copy-engine slab kernel
  } else if (S > 512 &&
             (dt == TVC_E4M3 || ((dt == TVC_BF16 || dt == TVC_F16) && s.v % 2 == 0) ||
              (dt == TVC_F32 && s.v % 4 == 0)) &&
             aligned(A, 16)) {
    // Large slabs: staged 16-byte pieces (see the kernel).  Measured on
    // 4096x4096x16 mode 1: BF16 3.5 TB/s, E4M3 2.1, FP32 5.0 (the per-warp
    // slab kernel: 2.2, 0.54 and 4.9; FP32 on 16384x8192x8: 5.5 against
    // 5.0); 2-byte types with odd v (one column per thread) measured below
    // the per-warp kernel and keep it, as do FP32 with v % 4 != 0 and FP64.
    p.kind = K_SLAB_ASYNC;
    // columns per thread: W elements from one shared-memory load (a tile
    // starts at element (i n_k + j) v, so v % W == 0 keeps the load aligned)
    p.vec = (s.v % 4 == 0) ? 4 : (s.v % 2 == 0) ? 2 : 1;
    const int64_t J = kSlabTile / (s.v * (int64_t)es);
    const int64_t target_blocks = (int64_t)sms * 4;
    int64_t splits = 1;
    if (s.u < target_blocks) splits = std::min(ceil_div(target_blocks, s.u), std::max<int64_t>(1, s.nk / (2 * J)));
    p.chunk = ceil_div(ceil_div(s.nk, splits), J) * J;
    p.splits = ceil_div(s.nk, p.chunk);
    p.grid = dim3((unsigned)s.u, (unsigned)p.splits);
  } else if (S > 512) {
    p.kind = K_SLAB;
    p.G = (int)(32 / s.v);
    p.g = p.G * (int)s.v;
    const int64_t target_warps = (int64_t)sms * 64;
    int64_t splits = 1;
    if (s.u < target_warps) splits = std::min(ceil_div(target_warps, s.u), std::max<int64_t>(1, s.nk / (16 * p.G)));
    p.chunk = ceil_div(ceil_div(s.nk, splits), p.G) * p.G;
    p.splits = ceil_div(s.nk, p.chunk);
    p.grid = dim3((unsigned)ceil_div(s.u, kWarpsPerBlock), (unsigned)p.splits);
  } else if (aligned(A, 16)) {
    // Small slabs, persistent double-buffered tiles (see the kernel).
    plan_tile_async(p, s, es, f64acc, sms);
  } else {
    p.kind = K_TILE;
    int64_t R = std::min<int64_t>(kThreads / s.v, (int64_t)(48 * 1024) / (int64_t)(S * es));
    R = std::max<int64_t>(1, std::min<int64_t>(R, s.u));
    if (R >= 16) R = R / 16 * 16;
    p.R = (int)R;
    p.vec16 = aligned(A, 16) && (((size_t)R * S * es) % 16 == 0);
    const size_t tile_bytes = ((size_t)R * S * es + 15) / 16 * 16;
    p.smem = tile_bytes + (size_t)s.nk * 8;
    p.splits = 1;
    p.chunk = s.nk;
    p.grid = dim3((unsigned)ceil_div(s.u, R), 1);
  }
  if (f64acc) p.ws_xs = align_up((size_t)s.nk * sizeof(XSplit), 256);
  if (p.xs_shift) p.ws_xs += align_up((size_t)(s.nk + 2) * sizeof(XSplit), 256);
  if (p.splits > 1) p.ws_partial = align_up((size_t)p.splits * s.uv * vec_size(dt), 256);
  p.ws_total = p.ws_xs + p.ws_partial;
  return p;
}

size_t tvc_ws_bytes(const Shape& s, tvc_dtype dt, const void* A) { return make_plan(s, dt, A).ws_total; }

template <tvc_dtype DT, int VEC>
static void launch_rows_vec(const Plan& p, const TvcArgs<DT>& a, cudaStream_t st) {
  switch (p.G) {
    case 2: tvc_rows_kernel<DT, VEC, 2><<<p.grid, kThreads, 0, st>>>(a); break;
    case 4: tvc_rows_kernel<DT, VEC, 4><<<p.grid, kThreads, 0, st>>>(a); break;
    case 8: tvc_rows_kernel<DT, VEC, 8><<<p.grid, kThreads, 0, st>>>(a); break;
    case 16: tvc_rows_kernel<DT, VEC, 16><<<p.grid, kThreads, 0, st>>>(a); break;
    default: tvc_rows_kernel<DT, VEC, 32><<<p.grid, kThreads, 0, st>>>(a); break;
  }
}

template <tvc_dtype DT>
static void launch_rows(const Plan& p, const TvcArgs<DT>& a, cudaStream_t st) {
  if constexpr (DT == TVC_F64) {
    if (p.xs_shift) tvc_rows_kernel<DT, 2, 32, true><<<p.grid, kThreads, 0, st>>>(a);  // the planner sets G = 32
    else if (p.vec == 2) launch_rows_vec<DT, 2>(p, a, st);
    else launch_rows_vec<DT, 1>(p, a, st);
  } else if constexpr (DT == TVC_F32 || DT == TVC_F32D) {
    if (p.vec == 4) launch_rows_vec<DT, 4>(p, a, st);
    else launch_rows_vec<DT, 1>(p, a, st);
  } else if constexpr (sizeof(typename Elem<DT>::T) == 2) {  // BF16, F16
    if (p.vec == 8) launch_rows_vec<DT, 8>(p, a, st);
    else if (p.vec == 2) launch_rows_vec<DT, 2>(p, a, st);
    else launch_rows_vec<DT, 1>(p, a, st);
  } else {
    if (p.vec == 16) launch_rows_vec<DT, 16>(p, a, st);
    else if (p.vec == 4) launch_rows_vec<DT, 4>(p, a, st);
    else launch_rows_vec<DT, 1>(p, a, st);
  }
}

template <tvc_dtype DT, int VEC, int RB>
static void launch_rows_multi_rb(const Plan& p, const TvcArgs<DT>& a, cudaStream_t st) {
  if (p.unr == 2) tvc_rows_multi_kernel<DT, VEC, RB, 2><<<p.grid, kThreads, 0, st>>>(a);
  else tvc_rows_multi_kernel<DT, VEC, RB, 1><<<p.grid, kThreads, 0, st>>>(a);
}

template <tvc_dtype DT>
static void launch_rows_multi(const Plan& p, const TvcArgs<DT>& a, cudaStream_t st) {
  if constexpr (!kF64Acc<DT>) {
    constexpr int VEC = 16 / (int)sizeof(typename Elem<DT>::T);
    if (p.rb == 2) launch_rows_multi_rb<DT, VEC, 2>(p, a, st);
    else if (p.rb == 8) launch_rows_multi_rb<DT, VEC, 8>(p, a, st);
    else launch_rows_multi_rb<DT, VEC, 4>(p, a, st);
  }
}

template <tvc_dtype DT, int VEC>
static void launch_rows_short_vec(const Plan& p, const TvcArgs<DT>& a, cudaStream_t st) {
  if (p.nst == 2) tvc_rows_short_kernel<DT, VEC, 2><<<p.grid, kThreads, 0, st>>>(a, p.G);
  else if (p.nst == 4) tvc_rows_short_kernel<DT, VEC, 4><<<p.grid, kThreads, 0, st>>>(a, p.G);
  else tvc_rows_short_kernel<DT, VEC, 8><<<p.grid, kThreads, 0, st>>>(a, p.G);
}

template <tvc_dtype DT>
static void launch_rows_short(const Plan& p, const TvcArgs<DT>& a, cudaStream_t st) {
  // The planner caps the vector width of short rows at 4 elements.
  if constexpr (DT == TVC_F64) {
    if (p.vec == 2) launch_rows_short_vec<DT, 2>(p, a, st);
    else launch_rows_short_vec<DT, 1>(p, a, st);
  } else {
    if (p.vec == 4) launch_rows_short_vec<DT, 4>(p, a, st);
    else if (p.vec == 2) launch_rows_short_vec<DT, 2>(p, a, st);
    else launch_rows_short_vec<DT, 1>(p, a, st);
  }
}

template <tvc_dtype DT>
static void launch_rows_tma(const Plan& p, const TvcArgs<DT>& a, cudaStream_t st) {
  RowsTmaParams prm;
  prm.R = p.R;
  prm.RW = p.RW;
  prm.S = p.S;
  prm.G = p.G;
  prm.nst = p.nst;
  prm.dq = p.dq;
  prm.ntiles = p.ntiles;
  prm.tile_bytes = p.tile_bytes;
  auto go = [&](auto kern) {
    opt_in_smem(reinterpret_cast<const void*>(kern), 200 * 1024);
    kern<<<p.grid, kTmaThreads, p.smem, st>>>(a, prm);
  };
  const bool n4 = p.nst <= 4;
  // The planner sends only FP32 and the narrow types here (FP64 rows are
  // faster in the register kernels).
  if constexpr (!kF64Acc<DT>) {
    if (p.vec == 4) n4 ? go(tvc_rows_tma_kernel<DT, 4, 4>) : go(tvc_rows_tma_kernel<DT, 4, 8>);
    else if (p.vec == 2) n4 ? go(tvc_rows_tma_kernel<DT, 2, 4>) : go(tvc_rows_tma_kernel<DT, 2, 8>);
    else n4 ? go(tvc_rows_tma_kernel<DT, 1, 4>) : go(tvc_rows_tma_kernel<DT, 1, 8>);
  }
}

template <tvc_dtype DT, int VEC, int DQ>
static void launch_rows_f64s_dq(const Plan& p, const TvcArgs<DT>& a, cudaStream_t st) {
  switch (p.G) {
    case 1: tvc_rows_f64_slots_kernel<DT, VEC, 1, DQ><<<p.grid, kThreads, 0, st>>>(a); break;
    case 2: tvc_rows_f64_slots_kernel<DT, VEC, 2, DQ><<<p.grid, kThreads, 0, st>>>(a); break;
    case 4: tvc_rows_f64_slots_kernel<DT, VEC, 4, DQ><<<p.grid, kThreads, 0, st>>>(a); break;
    case 8: tvc_rows_f64_slots_kernel<DT, VEC, 8, DQ><<<p.grid, kThreads, 0, st>>>(a); break;
    case 16: tvc_rows_f64_slots_kernel<DT, VEC, 16, DQ><<<p.grid, kThreads, 0, st>>>(a); break;
    default: tvc_rows_f64_slots_kernel<DT, VEC, 32, DQ><<<p.grid, kThreads, 0, st>>>(a); break;
  }
}

// Share (of 4 unrolled steps) of the FP64 short-row products sent to the
// DFMA pipe (exact FP64 products beside the float-float ones): 2 (measured:
// 128-element rows 5.45 -> 5.77 TB/s, 40-element rows unchanged).
constexpr int kSlotsDfmaSteps = 2;

template <tvc_dtype DT, int VEC>
static void launch_rows_f64s_vec(const Plan& p, const TvcArgs<DT>& a, cudaStream_t st) {
  if constexpr (DT == TVC_F64) launch_rows_f64s_dq<DT, VEC, kSlotsDfmaSteps>(p, a, st);
  else launch_rows_f64s_dq<DT, VEC, 0>(p, a, st);
}

template <tvc_dtype DT>
static bool launch_main(const Plan& p, const TvcArgs<DT>& a, cudaStream_t st) {
  switch (p.kind) {
    case K_COLS: {
      if constexpr (DT == TVC_F64) {
        if (p.vec == 2) {
          tvc_cols_kernel<DT, 2, 0><<<p.grid, kThreads, 0, st>>>(a);
        } else {
          tvc_cols_kernel<DT, 1, 0><<<p.grid, kThreads, 0, st>>>(a);
        }
      } else if constexpr (DT == TVC_F32 || DT == TVC_F32D) {
        if (p.vec == 4) tvc_cols_kernel<DT, 4, 0><<<p.grid, kThreads, 0, st>>>(a);
        else tvc_cols_kernel<DT, 1, 0><<<p.grid, kThreads, 0, st>>>(a);
      } else if constexpr (sizeof(typename Elem<DT>::T) == 2) {  // BF16, F16
        if (p.vec == 8) tvc_cols_async_kernel<DT, 8><<<p.grid, kThreads, 0, st>>>(a);
        else if (p.vec == 2) tvc_cols_kernel<DT, 2, 0><<<p.grid, kThreads, 0, st>>>(a);
        else tvc_cols_kernel<DT, 1, 0><<<p.grid, kThreads, 0, st>>>(a);
      } else {
        if (p.vec == 16) tvc_cols_async_kernel<DT, 16><<<p.grid, kThreads, 0, st>>>(a);
        else if (p.vec == 4) tvc_cols_kernel<DT, 4, 0><<<p.grid, kThreads, 0, st>>>(a);
        else tvc_cols_kernel<DT, 1, 0><<<p.grid, kThreads, 0, st>>>(a);
      }
      break;
    }
    case K_ROWS:
      launch_rows<DT>(p, a, st);
      break;
    case K_ROWS_MULTI:
      launch_rows_multi<DT>(p, a, st);
      break;
    case K_ROWS_SHORT:
      launch_rows_short<DT>(p, a, st);
      break;
    case K_ROWS_TMA:
      launch_rows_tma<DT>(p, a, st);
      break;
    case K_ROWS_F64S:
      if constexpr (DT == TVC_F64) {
        if (p.vec == 2) launch_rows_f64s_vec<DT, 2>(p, a, st);
        else launch_rows_f64s_vec<DT, 1>(p, a, st);
      } else if constexpr (DT == TVC_F32D) {
        if (p.vec == 4) launch_rows_f64s_vec<DT, 4>(p, a, st);
        else launch_rows_f64s_vec<DT, 1>(p, a, st);
      }
      break;
    case K_SLAB:
      if (slab_unroll(DT) == 16) tvc_slab_kernel<DT, 16><<<p.grid, kThreads, 0, st>>>(a, p.g, p.G);
      else tvc_slab_kernel<DT, 8><<<p.grid, kThreads, 0, st>>>(a, p.g, p.G);
      break;
    case K_SLAB_ASYNC:
      if constexpr (DT == TVC_F32) {
        tvc_slab_async_kernel<DT, 4><<<p.grid, kThreads, 0, st>>>(a);
      } else if constexpr (kNarrow<DT>) {
        if (p.vec == 4) tvc_slab_async_kernel<DT, 4><<<p.grid, kThreads, 0, st>>>(a);
        else if (p.vec == 2) tvc_slab_async_kernel<DT, 2><<<p.grid, kThreads, 0, st>>>(a);
        else tvc_slab_async_kernel<DT, 1><<<p.grid, kThreads, 0, st>>>(a);
      }
      break;
    case K_TILE_ASYNC: {
      opt_in_smem(reinterpret_cast<const void*>(tvc_tile_async_kernel<DT>), 200 * 1024);
      tvc_tile_async_kernel<DT><<<p.grid, kThreads, p.smem, st>>>(a, p.R, p.ntiles, p.vec16);
      break;
    }
    case K_F64_TILE:
      if constexpr (DT == TVC_F64) return f64tile_launch(a, p.ft, p.grid, st);
      break;
    case K_SLAB_TILE:
      if constexpr (DT == TVC_F32 || DT == TVC_BF16 || DT == TVC_F16 || DT == TVC_E4M3)
        slabtile_launch(a, p.st, p.grid, st);
      break;
    case K_TILE: {
      opt_in_smem(reinterpret_cast<const void*>(tvc_tile_kernel<DT>), 64 * 1024);
      tvc_tile_kernel<DT><<<p.grid, kThreads, p.smem, st>>>(a, p.R, p.vec16);
      break;
    }
  }
  return true;
}

template <tvc_dtype DT>
static tvc_status run(const void* A, const Shape& s, const void* x, void* y, const float* scales, double alpha,
                      double beta, void* ws, const Plan& p, cudaStream_t st, const int* done) {
  TvcArgs<DT> a;
  a.A = static_cast<const typename Elem<DT>::T*>(A);
  a.x = x;
  a.xs = nullptr;
  a.xs1 = nullptr;
  a.scales = scales;
  a.y = y;
  a.partial = nullptr;
  a.u = s.u;
  a.nk = s.nk;
  a.v = s.v;
  a.uv = s.uv;
  a.upi0 = s.upi0 > 0 ? s.upi0 : 1;
  a.chunk = p.chunk;
  a.splits = p.splits;
  a.mode0 = s.mode == 0;
  a.plain = (p.splits == 1 && alpha == 1.0 && beta == 0.0) ? 1 : 0;
  a.alpha = alpha;
  a.beta = beta;
  a.done = done;
  a.vmag = 0;
  a.vsh = -1;
  if (s.uv < ((int64_t)1 << 32) && s.v < ((int64_t)1 << 32)) div_magic((uint32_t)s.v, &a.vmag, &a.vsh);
  char* w = static_cast<char*>(ws);
  if (kF64Acc<DT>) {
    a.xs = reinterpret_cast<const XSplit*>(w);
    XSplit* xs1 = p.xs_shift ? reinterpret_cast<XSplit*>(w + align_up((size_t)s.nk * sizeof(XSplit), 256)) : nullptr;
    a.xs1 = xs1;
    const int blocks = (int)std::min<int64_t>(ceil_div(s.nk, 256), 4096);
    tvc_split_x_kernel<<<blocks, 256, 0, st>>>(static_cast<const double*>(x), reinterpret_cast<XSplit*>(w), xs1,
                                               s.nk, done);
  }
  if (p.splits > 1) a.partial = w + p.ws_xs;
  if (!launch_main<DT>(p, a, st)) return TVC_ERR_UNSUPPORTED;
  count_launches((kF64Acc<DT> ? 1 : 0) + 1 + (p.splits > 1 ? 1 : 0));
  if (p.splits > 1) {
    using V = typename Elem<DT>::V;
    const int blocks = (int)std::min<int64_t>(ceil_div(s.uv, 256), 8192);
    tvc_reduce_kernel<V><<<blocks, 256, 0, st>>>(static_cast<const V*>(a.partial), static_cast<V*>(y), s.uv,
                                                 p.splits, alpha, beta, done);
  }
  return cuda_status(cudaGetLastError());
}

tvc_status tvc_launch(const void* A, const Shape& s, const void* x, void* y, tvc_dtype dt, const float* scales,
                      double alpha, double beta, void* ws, size_t ws_bytes, cudaStream_t stream, const int* done) {
  const Plan p = make_plan(s, dt, A);
  if (p.ws_total > 0 && (ws == nullptr || ws_bytes < p.ws_total)) return TVC_ERR_WORKSPACE;
  switch (dt) {
    case TVC_F64: return run<TVC_F64>(A, s, x, y, nullptr, alpha, beta, ws, p, stream, done);
    case TVC_F32: return run<TVC_F32>(A, s, x, y, nullptr, alpha, beta, ws, p, stream, done);
    case TVC_BF16: return run<TVC_BF16>(A, s, x, y, scales, alpha, beta, ws, p, stream, done);
    case TVC_E4M3: return run<TVC_E4M3>(A, s, x, y, scales, alpha, beta, ws, p, stream, done);
    case TVC_F16: return run<TVC_F16>(A, s, x, y, scales, alpha, beta, ws, p, stream, done);
    case TVC_F32D: return run<TVC_F32D>(A, s, x, y, scales, alpha, beta, ws, p, stream, done);
  }
  return TVC_ERR_INVALID_ARG;
}

static tvc_status validate(const void* A, int order, const int64_t* dims, int mode, const void* x, void* y,
                           int dtype, Shape* s) {
  if (!valid_dtype(dtype)) return TVC_ERR_INVALID_ARG;
  tvc_status st = make_shape(order, dims, mode, s);
  if (st != TVC_OK) return st;
  if (!A || !x || !y) return TVC_ERR_INVALID_ARG;
  const size_t es = elem_size((tvc_dtype)dtype), vs = vec_size((tvc_dtype)dtype);
  if (!aligned(A, es) || !aligned(x, vs) || !aligned(y, vs)) return TVC_ERR_INVALID_ARG;
  return TVC_OK;
}

}  // namespace tvcg

using namespace tvcg;

extern "C" tvc_status tvc_device_error(int* code_out, int clear) {
  int v = 0, w = 0;
  if (cudaMemcpyFromSymbol(&v, g_tvc_device_error, sizeof(int)) != cudaSuccess) return TVC_ERR_CUDA;
  if (clear) {
    const int z = 0;
    if (cudaMemcpyToSymbol(g_tvc_device_error, &z, sizeof(int)) != cudaSuccess) return TVC_ERR_CUDA;
  }
  if (tmc_tc_device_error(&w, clear) != TVC_OK) return TVC_ERR_CUDA;
  if (v == 0 && w != 0) v = 10 + w;  // the tensor-core TMC kernel's waits
  if (f64tile_device_error(&w, clear) != TVC_OK) return TVC_ERR_CUDA;
  if (v == 0 && w != 0) v = 20 + w;  // the FP64 tile kernel's waits
  if (slabtile_device_error(&w, clear) != TVC_OK) return TVC_ERR_CUDA;
  if (v == 0 && w != 0) v = 30 + w;  // the slab tile kernel's waits
  if (code_out) *code_out = v;
  return v ? TVC_ERR_TIMEOUT : TVC_OK;
}

extern "C" size_t tvc_workspace_size(int order, const int64_t* dims, int mode, tvc_dtype dtype) {
  Shape s;
  if (!valid_dtype(dtype) || make_shape(order, dims, mode, &s) != TVC_OK) return 0;
  // The plan depends on the alignment of A, unknown here: return the largest
  // workspace over the alignments a tensor of this type can have.
  size_t need = 0;
  for (uintptr_t al = elem_size(dtype); al <= 256; al *= 2)
    need = std::max(need, tvc_ws_bytes(s, dtype, reinterpret_cast<const void*>(al)));
  return need;
}

extern "C" tvc_status tvc_ex(const void* A, int order, const int64_t* dims, int mode, const void* x, void* y,
                             tvc_dtype dtype, const float* slab_scales, double alpha, double beta, void* workspace,
                             size_t ws_bytes, tvc_stream_t stream) {
  Shape s;
  tvc_status st = validate(A, order, dims, mode, x, y, dtype, &s);
  if (st != TVC_OK) return st;
  return tvc_launch(A, s, x, y, dtype, slab_scales, alpha, beta, workspace, ws_bytes, (cudaStream_t)stream);
}

extern "C" tvc_status tvc(const void* A, int order, const int64_t* dims, int mode, const void* x, void* y,
                          tvc_dtype dtype, tvc_stream_t stream) {
  Shape s;
  tvc_status st = validate(A, order, dims, mode, x, y, dtype, &s);
  if (st != TVC_OK) return st;
  const cudaStream_t cs = (cudaStream_t)stream;
  const size_t need = tvc_ws_bytes(s, dtype, A);
  void* ws = nullptr;
  st = stream_scratch_alloc(need, cs, &ws);
  if (st != TVC_OK) return st;
  st = tvc_launch(A, s, x, y, dtype, nullptr, 1.0, 0.0, ws, need, cs);
  const tvc_status fr = stream_scratch_free(ws, cs);
  return st != TVC_OK ? st : fr;
}
