// Contraction of large slabs (1 < v < 32) whose rows are whole 16-byte
// pieces, for the FP32 accumulators (BF16, F16 and E4M3 storage with per-slab
// scales, and FP32): Y = alpha (A x_k x) + beta Y, Section 3 definition, Eq. 1
// form for one process.  v * sizeof(element) is 16, 32, 64 or 128 bytes
// (BF16 / F16 v = 8, 16; E4M3 v = 16; FP32 v = 4, 8, 16).
//
// The per-thread-staged slab kernel spent its issue slots on everything but
// the products (every thread issuing 16-byte copies of 8 KB tiles, two block
// barriers per tile, an x entry from global memory per row, and a serial sum
// over 64-128 row phases per slab).  Here:
//   * one producer lane copies tiles of up to 48 KB of consecutive rows of a
//     slab with cp.async.bulk into an NS-stage shared-memory ring (full /
//     empty mbarriers; every wait is bounded, and a block that saw a wait
//     give up records it and finishes with single-try waits, so it cannot
//     hang);
//   * eight consumer warps: thread t owns the 16-byte piece c = t mod CPR of
//     each row (CPR pieces per row) and the rows j = t div CPR (mod P),
//     P = 256 / CPR, decoding a whole piece per shared load (8 BF16 / F16,
//     16 E4M3 or 4 FP32 columns) and multiplying the columns pairwise with
//     the paired FP32 FMA; sums are folded into a compensated pair once per
//     tile (at most 64 rows per thread);
//   * at the end of a work item (one slab, or one split of its rows) the
//     threads of a piece are summed by a fixed xor-shuffle tree within each
//     warp, and the eight warps' sums in warp order: deterministic.
// E4M3 stays near 2.6 TB/s here (its decode takes 1.5 conversion
// instructions per element; an integer decode, three ALU operations per
// element, measured 2.0 TB/s: the kernel is latency-bound at 18 warps per
// SM, and the longer dependent chains cost more than the conversions).
#include <mutex>
#include <set>

#include "common.cuh"
#include "internal.h"
#include "tma.cuh"
#include "tvc_args.cuh"

namespace tvcg {

// Bounded waits that gave up (1: producer waited for a free stage, 2: a
// consumer waited for a tile, 3: the producer's final wait).
__device__ int g_slabtile_error = 0;

constexpr int kStWarps = 8;
constexpr int kStThreads = (kStWarps + 1) * kWarp;
constexpr long long kStWaitLimit = 4000000000LL;  // clock cycles (~2 s)

__device__ __forceinline__ uint64_t st_pk2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void st_upk2(uint64_t r, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ uint64_t st_fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

template <tvc_dtype DT>
__global__ void __launch_bounds__(kStThreads, 2) tvc_slabtile_kernel(const TvcArgs<DT> a,
                                                                      const SlabTileParams prm) {
  if (skip(a.done)) return;
  using E = Elem<DT>;
  using T = typename E::T;
  constexpr int es = (int)sizeof(T);
  constexpr int EPC = 16 / es;  // elements of a 16-byte piece
  constexpr int NP = EPC / 2;   // column pairs of a piece
  extern __shared__ __align__(128) unsigned char smraw[];
  const int NS = prm.NS, TR = prm.TR, CPR = prm.CPR;
  const int v = (int)a.v;
  const int P = (kStWarps * kWarp) / CPR;  // row phases
  const int row_bytes = v * es;            // 16 * CPR
  unsigned char* const stages = smraw;
  float* const part = reinterpret_cast<float*>(smraw + (size_t)NS * prm.stage_bytes);  // [kStWarps][v]
  uint64_t* const full = reinterpret_cast<uint64_t*>(smraw + (size_t)NS * prm.stage_bytes + prm.part_bytes);
  uint64_t* const empty = full + NS;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int q = 0; q < NS; q++) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], kStWarps);
    }
    mbar_fence_init();
  }
  __syncthreads();
  if (warp == kStWarps) {  // producer warp
    if (lane == 0) {
      bool failed = false;
      int k = 0;
      for (int64_t item = blockIdx.x; item < prm.nitems; item += gridDim.x) {
        const int64_t i = item / prm.splits, s = item - i * prm.splits;
        const int64_t jb = s * prm.chunk, je = min(a.nk, jb + prm.chunk);
        for (int64_t jt = jb; jt < je; jt += TR, k++) {
          const int st = k % NS;
          if (k >= NS && !mbar_wait(&empty[st], ((k / NS) - 1) & 1, &g_slabtile_error, 1, failed ? 0 : kStWaitLimit))
            failed = true;
          const uint32_t bytes = (uint32_t)(min((int64_t)TR, je - jt) * row_bytes);
          mbar_arrive_expect_tx(&full[st], bytes);
          tma_load_1d(stages + (size_t)st * prm.stage_bytes,
                      reinterpret_cast<const unsigned char*>(a.A) + ((i * a.nk + jt) * v) * es, bytes, &full[st]);
        }
      }
      // Never leave with copies in flight.
      for (int q = 0; q < NS && q < k; q++) {
        const int kk = k - 1 - q;
        mbar_wait(&full[kk % NS], (kk / NS) & 1, &g_slabtile_error, 3, 400000000LL);
      }
    }
    return;
  }
  const int c = tid % CPR, ph = tid / CPR;
  bool failed = false;
  int k = 0;
  for (int64_t item = blockIdx.x; item < prm.nitems; item += gridDim.x) {
    const int64_t i = item / prm.splits, s = item - i * prm.splits;
    const int64_t jb = s * prm.chunk, je = min(a.nk, jb + prm.chunk);
    float S[EPC], C[EPC];
#pragma unroll
    for (int e = 0; e < EPC; e++) {
      S[e] = 0.0f;
      C[e] = 0.0f;
    }
    for (int64_t jt = jb; jt < je; jt += TR, k++) {
      const int st = k % NS;
      if (!mbar_wait(&full[st], (k / NS) & 1, &g_slabtile_error, 2, failed ? 0 : kStWaitLimit)) failed = true;
      const int rows = (int)min((int64_t)TR, je - jt);
      const unsigned char* const tile = stages + (size_t)st * prm.stage_bytes + c * 16;
      uint64_t acc[NP];
#pragma unroll
      for (int q = 0; q < NP; q++) acc[q] = 0ull;
#pragma unroll 4
      for (int r = ph; r < rows; r += P) {
        const uint4 w = *reinterpret_cast<const uint4*>(tile + r * row_bytes);
        float val[EPC];
        const float xv = xval(a, jt + r);
        const uint64_t xx = st_pk2(xv, xv);
        E::decode16(w, val);
#pragma unroll
        for (int q = 0; q < NP; q++) acc[q] = st_fma2(st_pk2(val[2 * q], val[2 * q + 1]), xx, acc[q]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
      // fold this tile's sums (<= 64 rows per thread) into the compensated pairs
#pragma unroll
      for (int q = 0; q < NP; q++) {
        float lo, hi, t, err;
        st_upk2(acc[q], lo, hi);
        two_sum(S[2 * q], lo, t, err);
        S[2 * q] = t;
        C[2 * q] = __fadd_rn(C[2 * q], err);
        two_sum(S[2 * q + 1], hi, t, err);
        S[2 * q + 1] = t;
        C[2 * q + 1] = __fadd_rn(C[2 * q + 1], err);
      }
    }
    // the threads of one piece: lanes c, c + CPR, ... of each warp, then the
    // warps in order
#pragma unroll
    for (int e = 0; e < EPC; e++) {
      float r = __fadd_rn(S[e], C[e]);
      for (int m = CPR; m < kWarp; m <<= 1) r = __fadd_rn(r, __shfl_xor_sync(0xFFFFFFFFu, r, m));
      if (lane < CPR) part[warp * v + lane * EPC + e] = r;
    }
    named_barrier(1, kStWarps * kWarp);
    if (tid < v) {
      float sum = part[tid];
      for (int w = 1; w < kStWarps; w++) sum = __fadd_rn(sum, part[w * v + tid]);
      emit(a, s, i * a.v + tid, __fmul_rn(sum, out_scale(a, i)));
    }
    named_barrier(1, kStWarps * kWarp);  // part is rewritten by the next item
  }
}

size_t slabtile_smem_bytes(const SlabTileParams& prm) {
  return (size_t)prm.NS * prm.stage_bytes + prm.part_bytes + 2 * (size_t)prm.NS * sizeof(uint64_t);
}

template <tvc_dtype DT>
static void st_go(const TvcArgs<DT>& a, const SlabTileParams& prm, dim3 grid, cudaStream_t st) {
  static std::mutex mu;
  static std::set<int> done;
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(mu);
    if (done.insert(dev).second) {
      cudaFuncSetAttribute(tvc_slabtile_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      cudaFuncSetAttribute(tvc_slabtile_kernel<DT>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
  }
  tvc_slabtile_kernel<DT><<<grid, kStThreads, slabtile_smem_bytes(prm), st>>>(a, prm);
}

void slabtile_launch(const TvcArgs<TVC_F32>& a, const SlabTileParams& prm, dim3 grid, cudaStream_t st) {
  st_go<TVC_F32>(a, prm, grid, st);
}
void slabtile_launch(const TvcArgs<TVC_BF16>& a, const SlabTileParams& prm, dim3 grid, cudaStream_t st) {
  st_go<TVC_BF16>(a, prm, grid, st);
}
void slabtile_launch(const TvcArgs<TVC_F16>& a, const SlabTileParams& prm, dim3 grid, cudaStream_t st) {
  st_go<TVC_F16>(a, prm, grid, st);
}
void slabtile_launch(const TvcArgs<TVC_E4M3>& a, const SlabTileParams& prm, dim3 grid, cudaStream_t st) {
  st_go<TVC_E4M3>(a, prm, grid, st);
}

tvc_status slabtile_device_error(int* code_out, int clear) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_slabtile_error, sizeof(int)) != cudaSuccess) return TVC_ERR_CUDA;
  if (clear && v != 0) {
    const int z = 0;
    if (cudaMemcpyToSymbol(g_slabtile_error, &z, sizeof(int)) != cudaSuccess) return TVC_ERR_CUDA;
  }
  if (code_out) *code_out = v;
  return TVC_OK;
}

}  // namespace tvcg
