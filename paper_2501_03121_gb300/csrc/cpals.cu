// Building blocks of CP alternating least squares (Section 1 names the
// Khatri-Rao product and ALS for the canonical polyadic decomposition next
// to the TVC): the Khatri-Rao product of factor matrices and the
// matricized-tensor-times-Khatri-Rao product (MTTKRP)
//     M[i_k][r] = sum over all other indices of A[...] prod_{m != k} X_m[i_m][r].
//
// MTTKRP reads A once: with the matricized view u x n_k x v of Section 3,
// M[i_k][r] = sum_{i,l} A[i][i_k][l] KL[i][r] KR[l][r], where KL and KR are
// the Khatri-Rao products of the factors before and after mode k.  The
// larger of the two sides is contracted first by one tensor-matrix
// contraction over A (tmc.cu, with the transposed Khatri-Rao product as
// its R-row matrix), which leaves a small R x n_k x (other side) array;
// a second kernel contracts the other side with its Khatri-Rao rows in a
// fixed order.  Per-slab scales of narrow storage are folded into the
// Khatri-Rao rows (or, for k = 0 with u = 1, into the outputs), so the
// tensor pass runs with unit scales.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace tvcg {
namespace {

struct KrArgs {
  const void* U[TVC_MAX_ORDER];
  int64_t rows[TVC_MAX_ORDER];
  int count;
  int64_t R, nrows;
  int transposed;        // out[r][row] instead of out[row][r]
  const float* scales;   // nullable: row `row` times scales[row / per_slab]
  int64_t per_slab;
};

// out = U_0 (.) U_1 (.) ... (.) U_{count-1} (columnwise Kronecker product,
// row index with U_0's index most significant); count == 0 gives ones.
template <class V>
__global__ void khatri_rao_kernel(KrArgs a, V* __restrict__ out) {
  const int64_t n = a.nrows * a.R;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = a.transposed ? e % a.nrows : e / a.R;
    const int64_t r = a.transposed ? e / a.nrows : e % a.R;
    V p = 1;
    int64_t rem = row;
    for (int m = a.count - 1; m >= 0; m--) {
      const int64_t im = rem % a.rows[m];
      rem /= a.rows[m];
      p *= static_cast<const V*>(a.U[m])[im * a.R + r];
    }
    if (a.scales) p *= (V)a.scales[row / a.per_slab];
    out[e] = p;
  }
}

// M[i_k][r] = s(i_k) * sum_{q < K} T[(q / K2)*sq + (q % K2)*sq2 + i_k*sk + r*sr] * W[q*R + r];
// s(i_k) = scales[i_k] when given.  A block owns 32 consecutive outputs
// (e = i_k*R + r, one per lane) and its 8 warps split q (warp w takes
// q = w, w + 8, ...); the warps' sums are added in warp order (FP64, or
// compensated FP32 within a warp), a fixed order.
constexpr int kFinWarps = 8;

template <class V>
__global__ void __launch_bounds__(kFinWarps * 32) mttkrp_finish_kernel(const V* __restrict__ T,
                                                                       const V* __restrict__ W, V* __restrict__ M,
                                                                       int64_t nk, int64_t R, int64_t K, int64_t sq,
                                                                       int64_t sk, int64_t sr, const float* scales,
                                                                       int64_t K2, int64_t sq2) {
  __shared__ V part[kFinWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t n = nk * R;
  const int64_t e = (int64_t)blockIdx.x * 32 + lane;
  const bool act = e < n;
  const int64_t ik = act ? e / R : 0, r = act ? e - (e / R) * R : 0;
  const V* t = T + ik * sk + r * sr;
  V val = 0;
  if (act) {
    // q = q1 K2 + q2, advanced by kFinWarps without division
    int64_t q1 = w / K2, q2 = w - (w / K2) * K2;
    const int64_t d1 = kFinWarps / K2, d2 = kFinWarps - (kFinWarps / K2) * K2;
    if constexpr (sizeof(V) == 8) {
      double s = 0.0;
      for (int64_t q = w; q < K; q += kFinWarps) {
        s = fma(t[q1 * sq + q2 * sq2], W[q * R + r], s);
        q1 += d1;
        q2 += d2;
        if (q2 >= K2) {
          q2 -= K2;
          q1++;
        }
      }
      val = s;
    } else {
      KahanF32 s;
      float blk = 0.0f;
      int c = 0;
      for (int64_t q = w; q < K; q += kFinWarps) {
        blk = __fmaf_rn(t[q1 * sq + q2 * sq2], W[q * R + r], blk);
        q1 += d1;
        q2 += d2;
        if (q2 >= K2) {
          q2 -= K2;
          q1++;
        }
        if (++c == 64) {
          s.add(blk);
          blk = 0.0f;
          c = 0;
        }
      }
      s.add(blk);
      val = s.value();
    }
  }
  part[w][lane] = val;
  __syncthreads();
  if (w == 0 && act) {
    V tot = part[0][lane];
    for (int q = 1; q < kFinWarps; q++) tot += part[q][lane];
    if (scales) tot *= (V)scales[ik];
    M[e] = tot;
  }
}

// Workspace plan of one MTTKRP.
constexpr size_t kKrL2Bytes = 16u << 20;  // contracted Khatri-Rao rows kept L2-sized

struct MkPlan {
  bool right = true;    // contract the modes after k first
  int64_t u = 1, nk = 1, v = 1, R = 1;
  int msplit = 0;       // right side: modes [msplit, d) are contracted by the pass over A
  int64_t va = 1, vb = 1;  // right side: v = va * vb (modes (k, msplit) and [msplit, d))
  size_t vs = 4;        // bytes per vector entry
  size_t off_kt = 0, off_kw = 0, off_t = 0, off_tmc = 0, total = 0;
  int vorder = 0;       // view of A handed to the tensor-matrix contraction
  int64_t vdims[3] = {1, 1, 1};
  int vmode = 0;
  size_t tmc_ws = 0;
  bool t_is_m = false;  // the contraction writes M directly
};

MkPlan mk_plan(const Shape& s, int64_t R, tvc_dtype dt) {
  MkPlan p;
  p.u = s.u;
  p.nk = s.nk;
  p.v = s.v;
  p.R = R;
  p.vs = vec_size(dt);
  p.right = s.v >= s.u;
  if (p.right) {
    // The pass over A contracts the trailing modes [msplit, d): all of the
    // modes after k when their transposed Khatri-Rao rows (R x v) fit the
    // L2-sized budget, else the longest suffix that does (at least the last
    // mode), so that the rows re-read by every block of rows stay in L2;
    // the middle modes (k, msplit) are left to the finishing contraction.
    p.msplit = s.mode + 1;
    p.vb = s.v;
    while (p.msplit < s.order - 1 && (size_t)R * (size_t)p.vb * p.vs > kKrL2Bytes) {
      p.vb /= s.dims[p.msplit];
      p.msplit++;
    }
    p.va = s.v / p.vb;
    // A as (n_0, u n_k va / n_0, vb) (or (n_k va, vb) for k = 0), contracted over vb
    if (s.mode == 0) {
      p.vorder = 2;
      p.vdims[0] = s.nk * p.va;
      p.vdims[1] = p.vb;
      p.vmode = 1;
    } else {
      p.vorder = 3;
      p.vdims[0] = s.n0;
      p.vdims[1] = s.u * s.nk * p.va / s.n0;
      p.vdims[2] = p.vb;
      p.vmode = 2;
    }
    p.t_is_m = s.mode == 0 && p.va == 1;  // nothing left to contract: the pass writes M
  } else {
    // A as (u, n_k v), contracted over u
    p.vorder = 2;
    p.vdims[0] = s.u;
    p.vdims[1] = s.nk * s.v;
    p.vmode = 0;
  }
  const int64_t kt = R * (p.right ? p.vb : s.u);         // transposed Khatri-Rao rows of the contracted side
  const int64_t kw = R * (p.right ? s.u * p.va : s.v);  // Khatri-Rao rows of what is left
  const int64_t t = p.t_is_m ? 0 : R * s.nk * (p.right ? s.u * p.va : s.v);
  p.tmc_ws = tmc_workspace_size(p.vorder, p.vdims, p.vmode, R, dt);
  p.off_kt = 0;
  p.off_kw = align_up(p.off_kt + (size_t)kt * p.vs, 256);
  p.off_t = align_up(p.off_kw + (size_t)kw * p.vs, 256);
  p.off_tmc = align_up(p.off_t + (size_t)t * p.vs, 256);
  p.total = p.off_tmc + p.tmc_ws;
  return p;
}

int fin_blocks(int64_t n) { return (int)((n + 31) / 32); }

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 16LL * device_sms())); }

template <class V>
tvc_status kr_launch(const void* const* mats, const int64_t* rows, int count, int64_t R, int transposed,
                     const float* scales, int64_t per_slab, void* out, cudaStream_t st) {
  KrArgs a{};
  a.count = count;
  a.R = R;
  a.nrows = 1;
  for (int m = 0; m < count; m++) {
    a.U[m] = mats[m];
    a.rows[m] = rows[m];
    a.nrows *= rows[m];
  }
  a.transposed = transposed;
  a.scales = scales;
  a.per_slab = per_slab > 0 ? per_slab : 1;
  khatri_rao_kernel<V><<<grid_for(a.nrows * R), 256, 0, st>>>(a, static_cast<V*>(out));
  count_launches(1);
  return cuda_status(cudaGetLastError());
}

template <class V>
tvc_status mttkrp_run(const void* A, const Shape& s, const void* const* factors, int64_t R, void* M, tvc_dtype dt,
                      const float* scales, char* ws, const MkPlan& p, cudaStream_t st) {
  const int k = s.mode;
  const bool narrow = (dt == TVC_BF16 || dt == TVC_E4M3 || dt == TVC_F16) && scales;
  void* KT = ws + p.off_kt;
  void* KW = ws + p.off_kw;
  void* T = p.t_is_m ? M : (void*)(ws + p.off_t);
  tvc_status rc;
  // Khatri-Rao rows: the contracted side transposed (R x side), the other
  // side plain (side x R); the side that holds mode 0 carries the scales
  // (rows of u lie in slab i / (u / n_0) for k > 0).
  const void* lo_m[TVC_MAX_ORDER];
  int64_t lo_r[TVC_MAX_ORDER];
  const void* hi_m[TVC_MAX_ORDER];
  int64_t hi_r[TVC_MAX_ORDER];
  int nlo = 0, nhi = 0;
  for (int m = 0; m < k; m++) {
    lo_m[nlo] = factors[m];
    lo_r[nlo++] = s.dims[m];
  }
  const int mfirst = p.right ? p.msplit : k + 1;  // right side: the middle modes go with the lower ones
  for (int m = k + 1; m < mfirst; m++) {
    lo_m[nlo] = factors[m];
    lo_r[nlo++] = s.dims[m];
  }
  for (int m = mfirst; m < s.order; m++) {
    hi_m[nhi] = factors[m];
    hi_r[nhi++] = s.dims[m];
  }
  const float* lo_scales = (narrow && k > 0) ? scales : nullptr;
  // rows of the lower Khatri-Rao product: (i, ia) with i in u; i lies in slab i / (u / n_0)
  const int64_t per_slab = k > 0 ? (s.u / s.n0) * (p.right ? p.va : 1) : 1;
  if (p.right) {
    rc = kr_launch<V>(hi_m, hi_r, nhi, R, 1, nullptr, 1, KT, st);
    if (rc != TVC_OK) return rc;
    if (!p.t_is_m) {
      rc = kr_launch<V>(lo_m, lo_r, nlo, R, 0, lo_scales, per_slab, KW, st);
      if (rc != TVC_OK) return rc;
    }
  } else {
    rc = kr_launch<V>(lo_m, lo_r, nlo, R, 1, lo_scales, per_slab, KT, st);
    if (rc != TVC_OK) return rc;
    rc = kr_launch<V>(hi_m, hi_r, nhi, R, 0, nullptr, 1, KW, st);
    if (rc != TVC_OK) return rc;
  }
  // the pass over A: T = A x_(contracted side) KT
  rc = tmc(A, p.vorder, p.vdims, p.vmode, KT, R, T, dt, nullptr, 1.0, 0.0, ws + p.off_tmc, p.tmc_ws, st);
  if (rc != TVC_OK) return rc;
  const float* out_scales = (narrow && k == 0) ? scales : nullptr;
  if (p.t_is_m && !out_scales) return TVC_OK;
  const V* Tv = static_cast<const V*>(T);
  const V* Wv = static_cast<const V*>(KW);
  if (p.right) {
    if (p.t_is_m) {
      // k = 0: M[i_0][r] = scale[i_0] * T[i_0][r] in place (one term of weight 1)
      rc = kr_launch<V>(nullptr, nullptr, 0, R, 0, nullptr, 1, KW, st);  // one row of ones
      if (rc != TVC_OK) return rc;
      mttkrp_finish_kernel<V><<<fin_blocks(p.nk * R), kFinWarps * 32, 0, st>>>(
          Tv, Wv, static_cast<V*>(M), p.nk, R, 1, 0, R, 1, out_scales, 1, 0);
    } else {
      // T: (u n_k va) x R, T[((i n_k + i_k) va + ia) R + r]; sum over q = (i, ia)
      // with the lower Khatri-Rao rows W[(i va + ia)][r]
      mttkrp_finish_kernel<V><<<fin_blocks(p.nk * R), kFinWarps * 32, 0, st>>>(
          Tv, Wv, static_cast<V*>(M), p.nk, R, p.u * p.va, p.nk * p.va * R, p.va * R, 1, out_scales, p.va, R);
    }
  } else {
    // T: R x (n_k v), T[r (n_k v) + i_k v + l]; sum over l with KR[l][r]
    mttkrp_finish_kernel<V><<<fin_blocks(p.nk * R), kFinWarps * 32, 0, st>>>(
        Tv, Wv, static_cast<V*>(M), p.nk, R, p.v, p.v, p.v, p.nk * p.v, out_scales, p.v, 1);
  }
  count_launches(1);
  return cuda_status(cudaGetLastError());
}

}  // namespace
}  // namespace tvcg

using namespace tvcg;

extern "C" tvc_status khatri_rao(const void* const* mats, int count, const int64_t* rows, int64_t R, void* out,
                                 tvc_dtype vdtype, tvc_stream_t stream) {
  if (count < 1 || count > TVC_MAX_ORDER || !mats || !rows || !out || R < 1) return TVC_ERR_INVALID_ARG;
  if (vdtype != TVC_F64 && vdtype != TVC_F32) return TVC_ERR_INVALID_ARG;
  int64_t n = 1;
  for (int m = 0; m < count; m++) {
    if (!mats[m] || rows[m] < 1 || !aligned(mats[m], vec_size(vdtype))) return TVC_ERR_INVALID_ARG;
    if (__builtin_mul_overflow(n, rows[m], &n) || n >= ((int64_t)1 << 40)) return TVC_ERR_INVALID_ARG;
  }
  int64_t nR;
  if (__builtin_mul_overflow(n, R, &nR) || nR >= ((int64_t)1 << 48)) return TVC_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  return vdtype == TVC_F64 ? kr_launch<double>(mats, rows, count, R, 0, nullptr, 1, out, st)
                           : kr_launch<float>(mats, rows, count, R, 0, nullptr, 1, out, st);
}

extern "C" size_t mttkrp_workspace_size(int order, const int64_t* dims, int mode, int64_t R, tvc_dtype dtype) {
  Shape s;
  if (!valid_dtype(dtype) || R < 1 || make_shape(order, dims, mode, &s) != TVC_OK) return 0;
  return mk_plan(s, R, dtype).total;
}

extern "C" tvc_status mttkrp(const void* A, int order, const int64_t* dims, int mode, const void* const* factors,
                             int64_t R, void* M, tvc_dtype dtype, const float* slab_scales, void* workspace,
                             size_t ws_bytes, tvc_stream_t stream) {
  if (!valid_dtype(dtype) || !A || !M || R < 1 || (order > 1 && !factors)) return TVC_ERR_INVALID_ARG;
  Shape s;
  tvc_status rc = make_shape(order, dims, mode, &s);
  if (rc != TVC_OK) return rc;
  const size_t vs = vec_size(dtype);
  for (int m = 0; m < order; m++)
    if (m != mode && (!factors[m] || !aligned(factors[m], vs))) return TVC_ERR_INVALID_ARG;
  if (!aligned(M, vs) || !aligned(A, elem_size(dtype))) return TVC_ERR_INVALID_ARG;
  int64_t t;
  if (__builtin_mul_overflow(s.uv, R, &t) || __builtin_mul_overflow(t, s.nk, &t) || t >= ((int64_t)1 << 56))
    return TVC_ERR_INVALID_ARG;
  if ((s.nk * R + 31) / 32 > 0x7FFFFFFF) return TVC_ERR_UNSUPPORTED;
  const MkPlan p = mk_plan(s, R, dtype);
  if (!workspace || ws_bytes < p.total) return TVC_ERR_WORKSPACE;
  if (!aligned(workspace, 256)) return TVC_ERR_INVALID_ARG;
  char* ws = static_cast<char*>(workspace);
  cudaStream_t st = (cudaStream_t)stream;
  return vs == 8 ? mttkrp_run<double>(A, s, factors, R, M, dtype, slab_scales, ws, p, st)
                 : mttkrp_run<float>(A, s, factors, R, M, dtype, slab_scales, ws, p, st);
}
