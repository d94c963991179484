// Adjoints of the contraction Y = A x_k x (the paper has no passage for them;
// they follow from the definition of Section 3 by differentiation):
//     gx[j]      = sum_{i,l} A[i][j][l] * gy[i][l]      (a contraction of A with
//                                                        the (d-1)-tensor gy)
//     gA[i][j][l] = gy[i][l] * x[j]  (+ beta * gA)     (a rank-1 write stream)
// in the u x n_k x v view of mode k.
//
// gx, v == 1 and k > 0: gx = (A viewed as u x n_k) x_0 gy, i.e. a TVC of
//   mode 0 on the unfolded view (the column kernel), with gy times the slab
//   scale for narrow storage.
// gx, otherwise: each thread owns VEC columns (i, l) of a column tile, keeps
//   gy[i][l] in registers and accumulates A[i][j][l]*gy[i][l] into one
//   register accumulator per row j of a chunk of JC rows; blocks walk the
//   column tiles persistently, then reduce their accumulators (warp
//   shuffles, then warps in a fixed order) to one partial row per block; a
//   second kernel adds the blocks' partials in a fixed order.  A is read
//   once; gy once per chunk of rows.
// gA: threads own a position and loop over the other index so that every
//   store is coalesced: columns (i, l) looping over j when v >= 32,
//   positions q = (j, l) of a slab looping over slabs i otherwise.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace tvcg {

constexpr int kBT = 256;  // threads per block
constexpr int kBW = kBT / kWarp;

template <tvc_dtype DT>
struct GradArgs {
  const typename Elem<DT>::T* A;
  const void* gy;   // vector type (FP64 / FP32)
  const float* scales;
  void* partial;    // [gridDim.x][nk] per chunk, vector type
  int64_t u, nk, v, uv, upi0;
  int mode0;
  int jc;           // rows per chunk (<= JC)
};

// ------------------------------------------------------------- gx, v >= 2

template <tvc_dtype DT, int VEC, int JC>
__global__ void __launch_bounds__(kBT) tvc_gradx_kernel(const GradArgs<DT> a) {
  using E = Elem<DT>;
  using T = typename E::T;
  using V = typename E::V;
  const int64_t j0 = (int64_t)blockIdx.y * a.jc;
  const int jn = (int)min((int64_t)a.jc, a.nk - j0);
  const int64_t ncol = a.uv / VEC;  // VEC divides v, hence uv
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ double red[kBW][JC];
  if constexpr (kF64Acc<DT>) {
    float s[JC], c[JC];
    double d[JC];
#pragma unroll
    for (int q = 0; q < JC; q++) {
      s[q] = 0.0f;
      c[q] = 0.0f;
      d[q] = 0.0;
    }
    int cnt = 0;
    for (int64_t col = (int64_t)blockIdx.x * kBT + threadIdx.x; col < ncol; col += (int64_t)gridDim.x * kBT) {
      const int64_t o = col * VEC;
      const int64_t i = o / a.v, l = o - i * a.v;
      const double* gyp = static_cast<const double*>(a.gy) + o;
      XSplit gs[VEC];
      double gd[VEC];
#pragma unroll
      for (int e = 0; e < VEC; e++) {
        gd[e] = __ldg(gyp + e);
        gs[e] = split_x(gd[e]);
      }
      const T* p = a.A + (i * a.nk + j0) * a.v + l;
      typename E::C r[JC][VEC];
#pragma unroll
      for (int q = 0; q < JC; q++)
        if (q < jn) E::template load<VEC>(p + (int64_t)q * a.v, r[q]);
#pragma unroll
      for (int q = 0; q < JC; q++)
        if (q < jn) {
#pragma unroll
          for (int e = 0; e < VEC; e++) df_mac(s[q], c[q], d[q], r[q][e], gyp + e, gs[e]);
        }
      if (++cnt == 32) {  // keep the float-float pairs short
#pragma unroll
        for (int q = 0; q < JC; q++) {
          d[q] += (double)s[q];
          d[q] += (double)c[q];
          s[q] = 0.0f;
          c[q] = 0.0f;
        }
        cnt = 0;
      }
    }
#pragma unroll
    for (int q = 0; q < JC; q++) {
      double t = (d[q] + (double)s[q]) + (double)c[q];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, off);
      if (lane == 0) red[warp][q] = t;
    }
  } else {
    AccF32<JC> acc;
    acc.init();
    int cnt = 0;
    for (int64_t col = (int64_t)blockIdx.x * kBT + threadIdx.x; col < ncol; col += (int64_t)gridDim.x * kBT) {
      const int64_t o = col * VEC;
      const int64_t i = o / a.v, l = o - i * a.v;
      const float* gyp = static_cast<const float*>(a.gy) + o;
      float g[VEC];
      float sc = 1.0f;
      if constexpr (kNarrow<DT>) {
        if (!a.mode0 && a.scales) sc = __ldg(a.scales + i / a.upi0);
      }
#pragma unroll
      for (int e = 0; e < VEC; e++) g[e] = __fmul_rn(__ldg(gyp + e), sc);
      const T* p = a.A + (i * a.nk + j0) * a.v + l;
      float r[JC][VEC];
#pragma unroll
      for (int q = 0; q < JC; q++)
        if (q < jn) E::template load<VEC>(p + (int64_t)q * a.v, r[q]);
#pragma unroll
      for (int q = 0; q < JC; q++)
        if (q < jn) {
#pragma unroll
          for (int e = 0; e < VEC; e++) acc.a[q] = __fmaf_rn(r[q][e], g[e], acc.a[q]);
        }
      if (++cnt == 16) {
        acc.fold();
        cnt = 0;
      }
    }
    acc.fold();
#pragma unroll
    for (int q = 0; q < JC; q++) {
      float t = acc.result(q);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, off);
      if (lane == 0) red[warp][q] = (double)t;
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < jn) {
    const int q = threadIdx.x;
    double t = 0.0;
    for (int w = 0; w < kBW; w++) t += red[w][q];
    V val = (V)t;
    if constexpr (kNarrow<DT>) {
      if (a.mode0 && a.scales) val = __fmul_rn(val, __ldg(a.scales + j0 + q));
    }
    static_cast<V*>(a.partial)[(int64_t)blockIdx.x * a.nk + j0 + q] = val;
  }
}

template <class V>
__global__ void tvc_gradx_reduce_kernel(const V* __restrict__ partial, V* __restrict__ gx, int64_t nk, int64_t nblk) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nk; j += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t b = 0; b < nblk; b++) s += (double)partial[b * nk + j];
    gx[j] = (V)s;
  }
}

// gy'[i] = gy[i] * scale[i / upi0] (narrow storage, v == 1, mode > 0).
__global__ void tvc_scale_gy_kernel(const float* __restrict__ gy, const float* __restrict__ scales, float* out,
                                    int64_t u, int64_t upi0) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < u; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = scales ? __fmul_rn(gy[i], scales[i / upi0]) : gy[i];
}

// ------------------------------------------------------------------- gA

template <class V>
__global__ void tvc_gradA_cols_kernel(const V* __restrict__ gy, const V* __restrict__ x, V* __restrict__ gA,
                                      int64_t uv, int64_t nk, int64_t v, double beta) {
  // thread = column (i, l); loop over j
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < uv; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = o / v, l = o - i * v;
    const V g = gy[o];
    V* p = gA + i * nk * v + l;
    for (int64_t j = 0; j < nk; j++, p += v) {
      V val = g * __ldg(x + j);
      if (beta != 0.0) val += (V)beta * *p;
      __stcs(p, val);
    }
  }
}

template <class V>
__global__ void tvc_gradA_slab_kernel(const V* __restrict__ gy, const V* __restrict__ x, V* __restrict__ gA,
                                      int64_t u, int64_t nk, int64_t v, double beta) {
  // thread = position q = j*v + l of a slab; loop over slabs i
  const int64_t S = nk * v;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < S; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = q / v, l = q - j * v;
    const V xj = x[j];
    for (int64_t i = blockIdx.y; i < u; i += gridDim.y) {
      V* p = gA + i * S + q;
      V val = __ldg(gy + i * v + l) * xj;
      if (beta != 0.0) val += (V)beta * *p;
      __stcs(p, val);
    }
  }
}

// ----------------------------------------------------------------- host --

namespace {

struct GxPlan {
  bool via_tvc = false;  // v == 1
  int vec = 1, jc = 8;
  int64_t nchunks = 1, nblk = 1;
  size_t ws_partial = 0, ws_gy = 0, ws_tvc = 0, total = 0;
  Shape view;  // v == 1: (u, nk) mode 0
};

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

GxPlan plan_gx(const Shape& s, tvc_dtype dt, const void* A) {
  GxPlan g;
  const size_t vs = vec_size(dt);
  if (s.v == 1 && s.mode > 0) {
    g.via_tvc = true;
    const int64_t d2[2] = {s.u, s.nk};
    make_shape(2, d2, 0, &g.view);
    const tvc_dtype tdt = (dt == TVC_F64) ? TVC_F64 : dt;
    g.ws_tvc = 0;
    for (uintptr_t al = elem_size(tdt); al <= 256; al *= 2)
      g.ws_tvc = std::max(g.ws_tvc, tvc_ws_bytes(g.view, tdt, reinterpret_cast<const void*>(al)));
    if (dt == TVC_BF16 || dt == TVC_E4M3 || dt == TVC_F16) g.ws_gy = align_up((size_t)s.u * 4, 256);
    g.total = align_up(g.ws_tvc, 256) + g.ws_gy;
    return g;
  }
  const int es = (int)elem_size(dt);
  const int cand = (dt == TVC_F64) ? 2 : ((dt == TVC_F32) ? 4 : 4);
  g.vec = 1;
  if (s.v % cand == 0 && aligned(A, (size_t)cand * es)) g.vec = cand;
  g.jc = (dt == TVC_F64 || dt == TVC_F32D) ? 8 : 16;
  g.nchunks = cdiv(s.nk, g.jc);
  const int64_t cols = s.uv / g.vec;
  const int64_t want = std::max<int64_t>(1, (int64_t)device_sms() * 4 / std::max<int64_t>(1, g.nchunks));
  g.nblk = std::max<int64_t>(1, std::min<int64_t>(cdiv(cols, kBT), want));
  g.ws_partial = align_up((size_t)g.nblk * s.nk * vs, 256);
  g.total = g.ws_partial;
  return g;
}

template <tvc_dtype DT, int VEC>
void launch_gx(const GxPlan& g, const GradArgs<DT>& a, cudaStream_t st) {
  dim3 grid((unsigned)g.nblk, (unsigned)g.nchunks);
  if constexpr (kF64Acc<DT>)
    tvc_gradx_kernel<DT, VEC, 8><<<grid, kBT, 0, st>>>(a);
  else
    tvc_gradx_kernel<DT, VEC, 16><<<grid, kBT, 0, st>>>(a);
}

template <tvc_dtype DT>
tvc_status run_gx(const GxPlan& g, const Shape& s, const void* A, const void* gy, void* gx, const float* scales,
                  void* ws, cudaStream_t st) {
  using V = typename Elem<DT>::V;
  GradArgs<DT> a;
  a.A = static_cast<const typename Elem<DT>::T*>(A);
  a.gy = gy;
  a.scales = scales;
  a.partial = ws;
  a.u = s.u;
  a.nk = s.nk;
  a.v = s.v;
  a.uv = s.uv;
  a.upi0 = s.upi0 > 0 ? s.upi0 : 1;
  a.mode0 = s.mode == 0;
  a.jc = g.jc;
  if (g.vec == 1)
    launch_gx<DT, 1>(g, a, st);
  else if (g.vec == 2)
    launch_gx<DT, 2>(g, a, st);
  else
    launch_gx<DT, 4>(g, a, st);
  const int blocks = (int)std::min<int64_t>(cdiv(s.nk, 256), 4096);
  tvc_gradx_reduce_kernel<V><<<blocks, 256, 0, st>>>(static_cast<const V*>(ws), static_cast<V*>(gx), s.nk, g.nblk);
  count_launches(2);
  return cuda_status(cudaGetLastError());
}

tvc_status grad_x(const Shape& s, const void* A, const void* gy, void* gx, tvc_dtype dt, const float* scales,
                  void* ws, size_t ws_bytes, cudaStream_t st) {
  const GxPlan g = plan_gx(s, dt, A);
  if (g.total > 0 && (ws == nullptr || ws_bytes < g.total)) return TVC_ERR_WORKSPACE;
  if (g.via_tvc) {
    char* w = static_cast<char*>(ws);
    const void* gyv = gy;
    if (dt == TVC_BF16 || dt == TVC_E4M3 || dt == TVC_F16) {
      float* gys = reinterpret_cast<float*>(w + align_up(g.ws_tvc, 256));
      const int blocks = (int)std::min<int64_t>(cdiv(s.u, 256), 4096);
      tvc_scale_gy_kernel<<<blocks, 256, 0, st>>>(static_cast<const float*>(gy), scales, gys, s.u,
                                                  s.upi0 > 0 ? s.upi0 : 1);
      count_launches(1);
      gyv = gys;
    }
    // Mode 0 of the unfolded u x n_k view, the slab scales already in gy.
    return tvc_launch(A, g.view, gyv, gx, dt, nullptr, 1.0, 0.0, ws, g.ws_tvc, st);
  }
  switch (dt) {
    case TVC_F64: return run_gx<TVC_F64>(g, s, A, gy, gx, scales, ws, st);
    case TVC_F32D: return run_gx<TVC_F32D>(g, s, A, gy, gx, scales, ws, st);
    case TVC_F32: return run_gx<TVC_F32>(g, s, A, gy, gx, scales, ws, st);
    case TVC_BF16: return run_gx<TVC_BF16>(g, s, A, gy, gx, scales, ws, st);
    case TVC_E4M3: return run_gx<TVC_E4M3>(g, s, A, gy, gx, scales, ws, st);
    case TVC_F16: return run_gx<TVC_F16>(g, s, A, gy, gx, scales, ws, st);
  }
  return TVC_ERR_INVALID_ARG;
}

template <class V>
tvc_status grad_A(const Shape& s, const V* x, const V* gy, V* gA, double beta, cudaStream_t st) {
  const int sms = device_sms();
  if (s.v >= 32) {
    const int blocks = (int)std::min<int64_t>(cdiv(s.uv, 256), (int64_t)sms * 16);
    tvc_gradA_cols_kernel<V><<<blocks, 256, 0, st>>>(gy, x, gA, s.uv, s.nk, s.v, beta);
  } else {
    const int64_t S = s.nk * s.v;
    const int64_t bx = std::min<int64_t>(cdiv(S, 256), (int64_t)sms * 16);
    const int64_t by = std::max<int64_t>(1, std::min<int64_t>(s.u, std::min<int64_t>(65535, (int64_t)sms * 16 / bx + 1)));
    tvc_gradA_slab_kernel<V><<<dim3((unsigned)bx, (unsigned)by), 256, 0, st>>>(gy, x, gA, s.u, s.nk, s.v, beta);
  }
  count_launches(1);
  return cuda_status(cudaGetLastError());
}

}  // namespace

size_t tvc_backward_ws_bytes(const Shape& s, tvc_dtype dt) {
  size_t need = 0;
  for (uintptr_t al = elem_size(dt); al <= 256; al *= 2)
    need = std::max(need, plan_gx(s, dt, reinterpret_cast<const void*>(al)).total);
  return need;
}

}  // namespace tvcg

using namespace tvcg;

extern "C" size_t tvc_backward_workspace_size(int order, const int64_t* dims, int mode, tvc_dtype dtype) {
  Shape s;
  if (!valid_dtype(dtype) || make_shape(order, dims, mode, &s) != TVC_OK) return 0;
  return tvc_backward_ws_bytes(s, dtype);
}

extern "C" tvc_status tvc_backward(const void* A, int order, const int64_t* dims, int mode, const void* x,
                                   const void* gy, void* gx, void* gA, tvc_dtype dtype, const float* slab_scales,
                                   double beta_A, void* workspace, size_t ws_bytes, tvc_stream_t stream) {
  if (!valid_dtype(dtype)) return TVC_ERR_INVALID_ARG;
  Shape s;
  tvc_status st = make_shape(order, dims, mode, &s);
  if (st != TVC_OK) return st;
  const size_t vs = vec_size(dtype);
  if (!gy || !aligned(gy, vs)) return TVC_ERR_INVALID_ARG;
  if (gx && (!A || !aligned(A, elem_size(dtype)) || !aligned(gx, vs))) return TVC_ERR_INVALID_ARG;
  if (gA && (!x || !aligned(x, vs) || !aligned(gA, vs))) return TVC_ERR_INVALID_ARG;
  cudaStream_t cs = (cudaStream_t)stream;
  if (gx) {
    st = grad_x(s, A, gy, gx, dtype, slab_scales, workspace, ws_bytes, cs);
    if (st != TVC_OK) return st;
  }
  if (gA) {
    if (vs == 8)  // FP64 vectors: TVC_F64, TVC_F32D
      st = grad_A<double>(s, static_cast<const double*>(x), static_cast<const double*>(gy), static_cast<double*>(gA),
                          beta_A, cs);
    else
      st = grad_A<float>(s, static_cast<const float*>(x), static_cast<const float*>(gy), static_cast<float*>(gA),
                         beta_A, cs);
  }
  return st;
}
