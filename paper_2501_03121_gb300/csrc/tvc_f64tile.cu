// FP64 contraction of small slabs and short rows, Y = alpha (A x_k x) + beta Y
// (Section 3 definition, Eq. 1 form for one process), for 1 <= v < 32 and
// slabs S = n_k * v small enough that several whole slabs make one tile.
//
// The FP64 products go through the float-float pieces of common.cuh (the
// FP64 pipe of this part is far too slow for one DFMA per element).  On these
// shapes the kernels that read A straight from global memory, or stage it
// with per-thread 16-byte copies, spent about 54 issued instructions per
// element, above the ~48 per element the SMs can issue at the HBM rate.
// This kernel trims everything around the arithmetic:
//   * one producer lane copies tiles of R whole slabs (contiguous bytes)
//     into an NS-stage shared-memory ring with cp.async.bulk (full / empty
//     mbarriers, every wait bounded); the 8 bytes that end a tile whose size
//     is not a multiple of 16 (only the last tile) are stored by that lane
//     before it arrives on the stage's barrier;
//   * eight consumer warps contract each tile: G lanes share an output
//     (lane L serves output L mod (32/G) of the warp's pass and the steps
//     j = p, p + G, p + 2G, ... with p = L div (32/G)); the steps go two at a
//     time through the paired FP32 instructions of sm_100 (add / sub / mul /
//     fma .f32x2): the low half of every pair register is the chain of even
//     steps and the high half the chain of odd steps, so both pieces of the
//     pair work on one output;
//   * the x pieces sit in shared memory as {xh_j0, xh_j1, xl_j0, xl_j1} per
//     step pair and lane part, the G parts of a step pair side by side (one
//     16-byte load per two steps, lanes of different parts on different
//     banks), zero past
//     n_k: the padded steps read a neighbouring element (or the slack after
//     the tile, filled with 1.0), whose product with a zero piece is exactly
//     zero;
//   * the window bits of the split are ORed over all steps and tested once
//     per output; an output that met an element (or x entry) outside the
//     window is recomputed from the tile with DFMA;
//   * FP64 instructions run only where a result leaves, on full warps: with
//     G > 1 the finished outputs are gathered into per-lane slots first;
//   * rows whose length is a multiple of 4 (their starts would fall on 8 or
//     fewer of the 16 shared-memory bank pairs) are copied as 2-D boxes two
//     elements wider than the row: the copy engine fills the extra columns
//     with zeros, which no step reads, and the padded row stride spreads
//     the rows over the banks;
//   * with one lane per output and rows that start on 16-byte boundaries,
//     the two steps of a pair are one 16-byte shared-memory load.
// No step is folded into FP64 inside the loop: a lane's chain has at most
// 32 products (the error model of common.cuh allows 64 per fold).
#include <mutex>
#include <set>

#include "common.cuh"
#include "internal.h"
#include "tma.cuh"
#include "tvc_args.cuh"

namespace tvcg {

// Bounded waits that gave up (1: producer waited for a free stage, 2: a
// consumer waited for a tile, 3: the producer's final wait).
__device__ int g_f64tile_error = 0;

constexpr int kFtWarps = 8;  // consumer warps
constexpr int kFtThreads = (kFtWarps + 1) * kWarp;

// ------------------------------------------------ paired FP32 operations
// One 64-bit register holds two binary32 values; each operation rounds
// both halves exactly as the scalar instruction would.

__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(uint64_t r, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Two steps (elements a0, a1 against the x pieces of steps j0, j1) of the
// float-float product and compensated sum of common.cuh, side by side:
// s, c are the pairs (even chain, odd chain) of running sums and errors.
// The window word of both elements is ORed into bad (tested >> 28 later).
__device__ __forceinline__ void ff_step2(uint64_t& s, uint64_t& c, uint32_t& bad, double a0, double a1,
                                         const ulonglong2 xx) {
  const uint32_t lo0 = (uint32_t)__double2loint(a0), hi0 = (uint32_t)__double2hiint(a0);
  const uint32_t lo1 = (uint32_t)__double2loint(a1), hi1 = (uint32_t)__double2hiint(a1);
  bad |= (hi0 * 2u - kDfWindowBase) | (hi1 * 2u - kDfWindowBase);
  // ah: the exponent rebiased (1023 -> 127) and the top 23 fraction bits
  const uint32_t hb0 = __funnelshift_l(lo0, hi0 - 0x38000000u, 3) | (hi0 & 0x80000000u);
  const uint32_t hb1 = __funnelshift_l(lo1, hi1 - 0x38000000u, 3) | (hi1 & 0x80000000u);
  const uint64_t ah = pk2(__uint_as_float(hb0), __uint_as_float(hb1));
  // al: the remaining 29 fraction bits times 2^(e - 1075), signed like a
  const uint64_t m = pk2(__uint2float_rn(lo0 & 0x1FFFFFFFu), __uint2float_rn(lo1 & 0x1FFFFFFFu));
  const uint64_t sc = pk2(__uint_as_float((hb0 & 0xFF800000u) - 0x1A000000u),
                          __uint_as_float((hb1 & 0xFF800000u) - 0x1A000000u));
  const uint64_t al = mul2(m, sc);
  // TwoProduct of the leading pieces (its exact error with two scalar FMAs:
  // the paired FMA form measured inexact here, 3e-8 instead of 1e-14
  // relative), then the cross terms
  const uint64_t p = mul2(ah, xx.x);
  float ah0, ah1, xh0, xh1, p0, p1;
  upk2(ah, ah0, ah1);
  upk2(xx.x, xh0, xh1);
  upk2(p, p0, p1);
  uint64_t e = pk2(__fmaf_rn(ah0, xh0, -p0), __fmaf_rn(ah1, xh1, -p1));
  e = fma2(ah, xx.y, e);
  e = fma2(al, xx.x, e);
  // TwoSum (Knuth) of the running sum and the leading product
  const uint64_t t = add2(s, p);
  const uint64_t bp = sub2(t, s);
  const uint64_t ap = sub2(t, bp);
  const uint64_t err = add2(sub2(s, ap), sub2(p, bp));
  s = t;
  c = add2(c, add2(err, e));
}

// Exact FP64 recomputation of one output from the tile (rare: an element or
// x entry outside the split window).
static __device__ __noinline__ double ft_redo(const double* base, int v, int nk, const double* x) {
  double d = 0.0;
  for (int j = 0; j < nk; j++) d = fma(base[(int64_t)j * v], x[j], d);
  return d;
}

__device__ __forceinline__ void ft_tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// G: lanes per output; V1: v == 1 (rows); W16: G == 1, rows starting on
// 16-byte boundaries in shared memory (both steps of a pair in one load).
// map: the 2-D view of the rows when prm.box_rows > 0 (padded rows).
template <int G, bool V1, bool W16>
__global__ void __launch_bounds__(kFtThreads, 2) tvc_f64tile_kernel(const TvcArgs<TVC_F64> a,
                                                                     const F64TileParams prm,
                                                                     const __grid_constant__ CUtensorMap map) {
  static_assert(!W16 || (G == 1 && V1), "paired loads need one lane per row");
  if (skip(a.done)) return;
  extern __shared__ __align__(128) unsigned char smraw[];
  constexpr int OPW = kWarp / G;         // outputs per warp pass
  constexpr int OPP = kFtWarps * OPW;    // outputs per block pass
  const int NS = prm.NS, R = prm.R, npairs = prm.npairs;
  const int nk = (int)a.nk;
  const int v = V1 ? 1 : (int)a.v;
  const int S = nk * v;        // elements of a slab in A
  const int SR = prm.srow;     // elements between slabs in a tile (S, or the padded row)
  unsigned char* const stages = smraw;
  ulonglong2* const xt = reinterpret_cast<ulonglong2*>(smraw + (size_t)NS * prm.stage_bytes);  // [npairs][G]
  uint64_t* const full = reinterpret_cast<uint64_t*>(xt + G * npairs);
  uint64_t* const empty = full + NS;
  __shared__ int x_out;  // some x entry outside the split window
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int q = 0; q < NS; q++) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], kFtWarps);
    }
    mbar_fence_init();
    x_out = 0;
  }
  __syncthreads();
  {
    int bad = 0;
    for (int e = tid; e < G * npairs; e += kFtThreads) {
      const int k = e / G, p = e - k * G;
      const int j0 = p + 2 * k * G, j1 = j0 + G;
      const XSplit x0 = j0 < nk ? ldxs(a.xs + j0) : XSplit{0.0f, 0.0f};
      const XSplit x1 = j1 < nk ? ldxs(a.xs + j1) : XSplit{0.0f, 0.0f};
      bad |= (x0.xh != x0.xh) | (x1.xh != x1.xh);
      ulonglong2 w;
      w.x = pk2(x0.xh, x1.xh);
      w.y = pk2(x0.xl, x1.xl);
      xt[e] = w;
    }
    if (bad) atomicOr(&x_out, 1);
    // Every stage starts as 1.0 (inside the window), so that padded steps
    // past the last tile element never force a redo.
    double* const st64 = reinterpret_cast<double*>(stages);
    const int n64 = (int)((size_t)NS * prm.stage_bytes / 8);
    for (int e = tid; e < n64; e += kFtThreads) st64[e] = 1.0;
    // order these generic stores before the copy engine's writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (warp == kFtWarps) {  // producer warp
    if (lane == 0) {
      int k = 0;
      for (int64_t t = blockIdx.x; t < prm.ntiles; t += gridDim.x, k++) {
        const int st = k % NS;
        if (k >= NS && !mbar_wait(&empty[st], ((k / NS) - 1) & 1, &g_f64tile_error, 1)) break;
        double* const dst = reinterpret_cast<double*>(stages + (size_t)st * prm.stage_bytes);
        if (prm.box_rows > 0) {
          // padded rows: R / box_rows boxes of box_rows x srow elements;
          // rows past u and columns past n_k arrive as zeros (counted bytes)
          mbar_arrive_expect_tx(&full[st], (uint32_t)(R * SR * 8));
          for (int b = 0; b < R; b += prm.box_rows)
            ft_tma_load_2d(dst + (size_t)b * SR, &map, 0, (int)(t * R + b), &full[st]);
          continue;
        }
        const int64_t rows = min((int64_t)R, a.u - t * R);
        const int64_t n = rows * S;                   // elements of this tile
        const uint32_t cb = (uint32_t)((n * 8) & ~(int64_t)15);  // bytes through the copy engine
        const double* const src = a.A + t * R * (int64_t)S;
        if ((int64_t)cb < n * 8) dst[n - 1] = src[n - 1];  // odd element count: the last one by hand
        if (cb > 0) {
          mbar_arrive_expect_tx(&full[st], cb);
          tma_load_1d(dst, src, cb, &full[st]);
        } else {
          mbar_arrive(&full[st]);
        }
      }
      // Never leave with copies in flight.
      for (int q = 0; q < NS && q < k; q++) {
        const int kk = k - 1 - q;
        mbar_wait(&full[kk % NS], (kk / NS) & 1, &g_f64tile_error, 3, 400000000LL);
      }
    }
    return;
  }
  const double* const x = static_cast<const double*>(a.x);
  const int oi = lane % OPW, p = lane / OPW;
  const ulonglong2* const xr = xt + p;  // this lane's pieces: xr[k * G]
  const uint32_t bad0 = x_out ? 0xFFFFFFFFu : 0u;
  // slots (G > 1): lane L holds the L-th finished output of the warp
  float slot_s = 0.0f, slot_c = 0.0f;
  double slot_d = 0.0;
  int64_t slot_o = -1;
  int slot_bad = 0, nslot = 0;
  auto flush = [&]() {
    const bool anyd = __any_sync(0xFFFFFFFFu, slot_bad != 0);
    if (slot_o >= 0) {
      const double yv = anyd ? (slot_d + (double)slot_s) + (double)slot_c : (double)slot_s + (double)slot_c;
      emit(a, 0, slot_o, yv);
    }
    slot_o = -1;
    slot_bad = 0;
    nslot = 0;
  };
  int k = 0;
  for (int64_t t = blockIdx.x; t < prm.ntiles; t += gridDim.x, k++) {
    const int st = k % NS;
    if (!mbar_wait(&full[st], (k / NS) & 1, &g_f64tile_error, 2)) break;
    const double* const tile = reinterpret_cast<const double*>(stages + (size_t)st * prm.stage_bytes);
    const int64_t i0 = t * R;
    const int rows = (int)min((int64_t)R, a.u - i0);
    const int nout = rows * v;
    for (int ob = 0; ob < nout; ob += OPP) {
      const int o = ob + warp * OPW + oi;
      const bool act = o < nout;
      const int oc = act ? o : 0;
      int r, l;
      if constexpr (V1) {
        r = oc;
        l = 0;
      } else {
        r = (int)div_v(a, oc);
        l = oc - r * v;
      }
      const double* const ob_base = tile + r * SR + l;  // element (r, 0, l)
      const double* tb = ob_base + p * v;
      uint64_t s2 = 0ull, c2 = 0ull;
      uint32_t badw = bad0;
      if constexpr (W16) {
#pragma unroll 4
        for (int kq = 0; kq < npairs; kq++) {
          const double2 a01 = *reinterpret_cast<const double2*>(tb);
          ff_step2(s2, c2, badw, a01.x, a01.y, xr[kq]);
          tb += 2;
        }
      } else if constexpr (V1) {
#pragma unroll 4
        for (int kq = 0; kq < npairs; kq++) {
          const double a0 = tb[0], a1 = tb[G];
          ff_step2(s2, c2, badw, a0, a1, xr[kq * G]);
          tb += 2 * G;
        }
      } else {
        const int stp = G * v;
#pragma unroll 4
        for (int kq = 0; kq < npairs; kq++) {
          const double a0 = tb[0], a1 = tb[stp];
          ff_step2(s2, c2, badw, a0, a1, xr[kq * G]);
          tb += 2 * stp;
        }
      }
      float sl, sh, cl, ch, s, c, e;
      upk2(s2, sl, sh);
      upk2(c2, cl, ch);
      two_sum(sl, sh, s, e);
      c = __fadd_rn(__fadd_rn(cl, ch), e);
#pragma unroll
      for (int m = OPW; m < kWarp; m <<= 1) {
        const float s_o = __shfl_xor_sync(0xFFFFFFFFu, s, m);
        const float c_o = __shfl_xor_sync(0xFFFFFFFFu, c, m);
        badw |= __shfl_xor_sync(0xFFFFFFFFu, badw, m);
        float tt, err;
        two_sum(s, s_o, tt, err);
        s = tt;
        c = __fadd_rn(c, __fadd_rn(c_o, err));
      }
      const int bad = (act && (badw >> 28) != 0) ? 1 : 0;
      double d = 0.0;
      if (bad && p == 0) {
        d = ft_redo(ob_base, v, nk, x);
        s = 0.0f;
        c = 0.0f;
      }
      if constexpr (G == 1) {
        const bool anyd = __any_sync(0xFFFFFFFFu, bad != 0);
        if (act) {
          const double yv = anyd ? (d + (double)s) + (double)c : (double)s + (double)c;
          emit(a, 0, i0 * v + o, yv);
        }
      } else {
        // move the OPW finished outputs (lanes 0 .. OPW-1) into slots nslot ..
        const int rel = lane - nslot;
        const bool mine = rel >= 0 && rel < OPW;
        const int srcl = mine ? rel : 0;
        const float ss = __shfl_sync(0xFFFFFFFFu, s, srcl);
        const float cc = __shfl_sync(0xFFFFFFFFu, c, srcl);
        const double dd = __shfl_sync(0xFFFFFFFFu, d, srcl);
        const int bb = __shfl_sync(0xFFFFFFFFu, bad, srcl);
        if (mine) {
          const int oo = ob + warp * OPW + rel;
          slot_s = ss;
          slot_c = cc;
          slot_d = dd;
          slot_bad = bb;
          slot_o = oo < nout ? i0 * v + oo : -1;
        }
        nslot += OPW;
        if (nslot == kWarp) flush();
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
  }
  if constexpr (G > 1) {
    if (nslot > 0) flush();
  }
}

size_t f64tile_smem_bytes(const F64TileParams& prm) {
  return (size_t)prm.NS * prm.stage_bytes + (size_t)prm.G * prm.npairs * sizeof(ulonglong2) +
         2 * (size_t)prm.NS * sizeof(uint64_t);
}

template <int G, bool V1, bool W16>
static void ft_go(const TvcArgs<TVC_F64>& a, const F64TileParams& prm, const CUtensorMap& map, dim3 grid,
                  size_t smem, cudaStream_t st) {
  static std::mutex mu;
  static std::set<int> done;
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(mu);
    if (done.insert(dev).second) {
      cudaFuncSetAttribute(tvc_f64tile_kernel<G, V1, W16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      cudaFuncSetAttribute(tvc_f64tile_kernel<G, V1, W16>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
  }
  tvc_f64tile_kernel<G, V1, W16><<<grid, kFtThreads, smem, st>>>(a, prm, map);
}

template <bool V1>
static void ft_dispatch(const TvcArgs<TVC_F64>& a, const F64TileParams& prm, const CUtensorMap& map, dim3 grid,
                        size_t smem, cudaStream_t st) {
  switch (prm.G) {
    case 1:
      if constexpr (V1) {
        if (prm.w16) {
          ft_go<1, true, true>(a, prm, map, grid, smem, st);
          break;
        }
      }
      ft_go<1, V1, false>(a, prm, map, grid, smem, st);
      break;
    case 2: ft_go<2, V1, false>(a, prm, map, grid, smem, st); break;
    case 4: ft_go<4, V1, false>(a, prm, map, grid, smem, st); break;
    case 8: ft_go<8, V1, false>(a, prm, map, grid, smem, st); break;
    case 16: ft_go<16, V1, false>(a, prm, map, grid, smem, st); break;
    default: ft_go<32, V1, false>(a, prm, map, grid, smem, st); break;
  }
}

bool f64tile_launch(const TvcArgs<TVC_F64>& a, const F64TileParams& prm, dim3 grid, cudaStream_t st) {
  const size_t smem = f64tile_smem_bytes(prm);
  CUtensorMap map{};
  if (prm.box_rows > 0) {
    // rows of n_k elements (row stride n_k * 8 bytes, a multiple of 16) read
    // as boxes of srow x box_rows; zero fill outside the tensor
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)a.nk, (cuuint64_t)a.u};
    const cuuint64_t strides[1] = {(cuuint64_t)a.nk * 8};
    const cuuint32_t box[2] = {(cuuint32_t)prm.srow, (cuuint32_t)prm.box_rows};
    const cuuint32_t estr[2] = {1, 1};
    if (fn(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(a.A), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  if (a.v == 1) ft_dispatch<true>(a, prm, map, grid, smem, st);
  else ft_dispatch<false>(a, prm, map, grid, smem, st);
  return true;
}

tvc_status f64tile_device_error(int* code_out, int clear) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_f64tile_error, sizeof(int)) != cudaSuccess) return TVC_ERR_CUDA;
  if (clear && v != 0) {
    const int z = 0;
    if (cudaMemcpyToSymbol(g_f64tile_error, &z, sizeof(int)) != cudaSuccess) return TVC_ERR_CUDA;
  }
  if (code_out) *code_out = v;
  return TVC_OK;
}

}  // namespace tvcg
