// Arguments of the TVC kernels and the store of one result, shared by the
// translation units that hold TVC kernels (tvc.cu, tvc_f64tile.cu,
// tvc_slabtile.cu).
#pragma once

#include "common.cuh"
#include "internal.h"

namespace tvcg {

template <tvc_dtype DT>
struct TvcArgs {
  const typename Elem<DT>::T* A;
  const void* x;        // FP64 for F64, FP32 otherwise
  const XSplit* xs;     // F64: split x (workspace)
  const XSplit* xs1;    // F64 rows of odd length: xs shifted by one entry (xs1[j + 1] = xs[j], zeros at both ends)
  const float* scales;  // narrow types, nullable
  void* y;
  void* partial;
  int64_t u, nk, v, uv, upi0, chunk, splits;
  int mode0;
  int plain;  // splits == 1, alpha == 1, beta == 0: y[o] = value
  double alpha, beta;
  const int* done;  // nullable: when *done != 0 the kernel returns at once
  uint32_t vmag;    // u*v < 2^32: o / v = (umulhi(o, vmag) + o) >> vsh (vsh < 0: divide)
  int vsh;
};

// Magic multiplier and shift of a 32-bit divisor d >= 1 (Granlund and
// Montgomery, division by invariant integers): for every 32-bit n,
// n / d = (umulhi(n, m) + n) >> s with s = ceil(log2 d) and
// m = floor(2^32 (2^s - d) / d) + 1, the sum taken in 64 bits.
inline void div_magic(uint32_t d, uint32_t* m, int* s) {
  int k = 0;
  while (k < 32 && (uint64_t(1) << k) < d) k++;
  *s = k;
  *m = (uint32_t)((((uint64_t)1 << 32) * ((uint64_t(1) << k) - d)) / d + 1);
}

// o / v for an output index o of the contraction (v the trailing size).
template <tvc_dtype DT>
__device__ __forceinline__ int64_t div_v(const TvcArgs<DT>& a, int64_t o) {
  if (a.vsh >= 0) {
    const uint32_t n = (uint32_t)o;
    return (int64_t)(((uint64_t)__umulhi(n, a.vmag) + n) >> a.vsh);
  }
  return o / a.v;
}

// Early exit of work queued behind a converged (or failed) power method.
__device__ __forceinline__ bool skip(const int* done) {
  return done != nullptr && *reinterpret_cast<const volatile int*>(done) != 0;
}

__device__ __forceinline__ XSplit ldxs(const XSplit* p) {
  float2 f = __ldg(reinterpret_cast<const float2*>(p));
  return XSplit{f.x, f.y};
}

// x entry of row j for the FP32 accumulators (slab scale folded in for k = 0).
template <tvc_dtype DT>
__device__ __forceinline__ float xval(const TvcArgs<DT>& a, int64_t j) {
  float xv = __ldg(static_cast<const float*>(a.x) + j);
  if constexpr (kNarrow<DT>) {
    if (a.mode0 && a.scales) xv = __fmul_rn(xv, __ldg(a.scales + j));
  }
  return xv;
}

// Scale of output row i (k > 0): all elements of an output share slab i / upi0.
template <tvc_dtype DT>
__device__ __forceinline__ float out_scale(const TvcArgs<DT>& a, int64_t i) {
  if constexpr (kNarrow<DT>) {
    if (!a.mode0 && a.scales) return __ldg(a.scales + i / a.upi0);
  }
  return 1.0f;
}

template <tvc_dtype DT>
__device__ __forceinline__ void emit(const TvcArgs<DT>& a, int64_t s, int64_t o,
                                     typename Elem<DT>::V val) {
  using V = typename Elem<DT>::V;
  if (a.plain) {
    static_cast<V*>(a.y)[o] = val;
  } else if (a.splits == 1) {
    V* y = static_cast<V*>(a.y);
    V r = (V)a.alpha * val;
    if (a.beta != 0.0) r += (V)a.beta * y[o];
    y[o] = r;
  } else {
    static_cast<V*>(a.partial)[s * a.uv + o] = val;
  }
}

// FP64 small slabs and short rows through the copy engine (tvc_f64tile.cu).
// A tile is R whole slabs (R*S elements, S = n_k*v, R*S even so that every
// tile starts on a 16-byte boundary; or R padded rows); G lanes share one output, each taking
// the products j = p, p + G, ... (2*npairs of them, zero x pieces past n_k).
struct F64TileParams {
  int R;                // slabs per tile
  int G;                // lanes per output (1, 2, 4, 8, 16 or 32)
  int NS;               // stages of the shared-memory ring
  int npairs;           // ceil(ceil(n_k / G) / 2)
  int64_t ntiles;       // ceil(u / R)
  uint32_t stage_bytes; // stride between stages: R*srow*8 plus slack for the padded reads
  int srow;             // elements between consecutive slabs of a tile in shared memory
  int box_rows;         // > 0: rows (v = 1) copied as 2-D boxes of box_rows x srow (srow > n_k)
  int w16;              // G == 1, v == 1, rows on 16-byte boundaries: paired 16-byte loads
};
// Shared memory of one block of that kernel for the given parameters.
size_t f64tile_smem_bytes(const F64TileParams& prm);
// Returns false (nothing launched) when the 2-D copy view cannot be made.
bool f64tile_launch(const TvcArgs<TVC_F64>& a, const F64TileParams& prm, dim3 grid, cudaStream_t st);
// Sticky error word of its bounded waits (cleared when clear != 0).
tvc_status f64tile_device_error(int* code_out, int clear);

// Large slabs whose rows are whole 16-byte pieces, FP32 accumulators
// (tvc_slabtile.cu): work items are (slab, split of its rows), tiles of TR
// rows; CPR = v * sizeof(element) / 16 pieces per row (1, 2, 4 or 8).
struct SlabTileParams {
  int TR;                // rows per tile
  int NS;                // stages of the shared-memory ring
  int CPR;               // 16-byte pieces per row
  int64_t nitems;        // u * splits
  int64_t splits, chunk; // splits of n_k and rows per split
  uint32_t stage_bytes;  // stride between stages
  uint32_t part_bytes;   // per-warp column sums (8 * v floats, rounded to 16 bytes)
};
size_t slabtile_smem_bytes(const SlabTileParams& prm);
void slabtile_launch(const TvcArgs<TVC_F32>& a, const SlabTileParams& prm, dim3 grid, cudaStream_t st);
void slabtile_launch(const TvcArgs<TVC_BF16>& a, const SlabTileParams& prm, dim3 grid, cudaStream_t st);
void slabtile_launch(const TvcArgs<TVC_F16>& a, const SlabTileParams& prm, dim3 grid, cudaStream_t st);
void slabtile_launch(const TvcArgs<TVC_E4M3>& a, const SlabTileParams& prm, dim3 grid, cudaStream_t st);
tvc_status slabtile_device_error(int* code_out, int clear);

}  // namespace tvcg
