// Higher-order power method (Section 3, "HOPM") in the three-buffer form of
// Algorithm 1 for one GPU (p = 1): Gauss-Seidel sweeps over the external
// modes j = 0 .. d-1, each computing z_j = A x_{m != j} x_m and x_j = z_j/||z_j||.
//
// Every sweep streams A exactly twice, both times with the column kernel of
// the TVC (the bandwidth-bound part):
//   j = 0:  T   = A x_1 x_1                     (Algorithm 1's first contraction)
//           z_0 = rows of T . (x_2 (x) ... (x) x_{d-1})
//   j = 1:  W_1 = A x_0 x_0                     (prefix cache)
//           z_1 = rows of W_1 . (x_2 (x) ... (x) x_{d-1})
//   j >= 2: W_j = W_{j-1} x_{j-1} x_{j-1}       (first remaining mode)
//           z_j = rows of W_j . (x_{j+1} (x) ... (x) x_{d-1})   (z_{d-1} = W_{d-1})
// The d-2 (resp. d-j-1) trailing contractions of each external iteration are
// fused into one pass over the small tensor against the outer product of
// the trailing vectors, so intermediate tensors beyond T and W_j are never
// written.  The norm, x_j, lambda (= ||z_{d-1}||, the value A(x_0,...,x_{d-1})
// reached at the end of a sweep), the stopping test and the status word are
// computed in FP64 by one device kernel; once the sweep has converged or
// failed, a device flag makes every queued kernel return at once, so the
// host can queue all sweeps without synchronising (and capture them in a
// CUDA graph).
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace tvcg {

// Device-resident state of one power-method run (in the workspace).
struct HopmState {
  double lam;       // lambda of the last completed sweep
  double lam_prev;  // lambda of the sweep before
  int sweeps;       // completed sweeps
  int status;       // tvc_status of the device side
  int done;         // 1 once converged or failed: later kernels return
  int pad;
};

__device__ __forceinline__ bool hskip(const HopmState* st) {
  return *reinterpret_cast<const volatile int*>(&st->done) != 0;
}

__global__ void hopm_init_kernel(HopmState* st) {
  st->lam = 0.0;
  st->lam_prev = 0.0;
  st->sweeps = 0;
  st->status = TVC_OK;
  st->done = 0;
  st->pad = 0;
}

// w[c] = prod_m x_m[i_m(c)] over nm trailing vectors (row-major digits of c),
// formed left to right in the vector precision V.
struct OuterArgs {
  int nm;
  int64_t dims[TVC_MAX_ORDER];
  const void* xs[TVC_MAX_ORDER];
};

template <class V>
__global__ void hopm_outer_kernel(V* __restrict__ w, int64_t n, OuterArgs oa, const HopmState* st) {
  if (hskip(st)) return;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = c;
    int64_t dig[TVC_MAX_ORDER];
    for (int m = oa.nm - 1; m >= 0; m--) {
      dig[m] = rem % oa.dims[m];
      rem /= oa.dims[m];
    }
    V acc = static_cast<const V*>(oa.xs[0])[dig[0]];
    for (int m = 1; m < oa.nm; m++) acc *= static_cast<const V*>(oa.xs[m])[dig[m]];
    w[c] = acc;
  }
}

// x_j = z / ||z||_2 with the norm in FP64 (fixed-order block reduction, so
// the result is reproducible).  For the last mode of a sweep it also sets
// lambda, counts the sweep and applies the stopping rule
//   stop when tol > 0, sweep >= 2 and |lambda_t - lambda_{t-1}| <= tol*lambda_t.
// A zero or non-finite norm sets the status, leaves x_j unchanged and stops.
constexpr int kNormThreads = 512;

template <class V>
__global__ void __launch_bounds__(kNormThreads) hopm_normalize_kernel(const V* __restrict__ z, V* __restrict__ xj,
                                                                     int64_t n, int last, double tol, HopmState* st,
                                                                     double* lam_out, int* sweeps_out,
                                                                     int* status_out, double* lam_hist) {
  if (hskip(st)) return;
  __shared__ double red[kNormThreads];
  double ss = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kNormThreads) {
    const double v = (double)z[i];
    ss = fma(v, v, ss);
  }
  red[threadIdx.x] = ss;
  __syncthreads();
  for (int off = kNormThreads / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  const double sigma = sqrt(red[0]);
  const bool finite = isfinite(sigma);
  const bool zero = (sigma == 0.0);
  if (finite && !zero) {
    for (int64_t i = threadIdx.x; i < n; i += kNormThreads) xj[i] = (V)((double)z[i] / sigma);
  }
  if (threadIdx.x == 0) {
    int status = TVC_OK;
    if (!finite) status = TVC_ERR_NONFINITE;
    else if (zero) status = TVC_ERR_ZERO_NORM;
    if (status != TVC_OK) {
      st->status = status;
      st->done = 1;
    } else if (last) {
      const int t = st->sweeps + 1;
      st->sweeps = t;
      st->lam_prev = st->lam;
      st->lam = sigma;
      if (lam_hist) lam_hist[t - 1] = sigma;
      const double scale = sigma > 1e-300 ? sigma : 1e-300;
      if (tol > 0.0 && t >= 2 && fabs(sigma - st->lam_prev) <= tol * scale) st->done = 1;
    }
    if (lam_out) *lam_out = st->lam;
    if (sweeps_out) *sweeps_out = st->sweeps;
    if (status_out) *status_out = st->status;
  }
}

// ---------------------------------------------------------------- host ----

namespace {

struct HopmPlan {
  int d = 0;
  int64_t dims[TVC_MAX_ORDER] = {};
  int64_t N = 0;
  size_t vs = 8;
  // workspace layout (byte offsets)
  size_t off_state = 0, off_bufA = 0, off_bufB = 0, off_w = 0, off_z = 0, off_tvc = 0, total = 0;
  size_t tvc_ws = 0;
};

Shape shape2(int64_t a, int64_t b, int mode) {
  Shape s;
  const int64_t d2[2] = {a, b};
  make_shape(2, d2, mode, &s);
  return s;
}

int64_t prod_range(const int64_t* dims, int lo, int hi) {
  int64_t p = 1;
  for (int i = lo; i < hi; i++) p *= dims[i];
  return p;
}

// The contractions one sweep issues, as (shape, dtype) pairs, for sizing.
template <class F>
void for_each_tvc(const HopmPlan& hp, tvc_dtype dt, F f) {
  const int d = hp.d;
  const int64_t* n = hp.dims;
  const tvc_dtype vdt = (dt == TVC_F64) ? TVC_F64 : TVC_F32;
  Shape s;
  if (d == 2) {
    make_shape(2, n, 1, &s);
    f(s, dt);
    make_shape(2, n, 0, &s);
    f(s, dt);
    return;
  }
  make_shape(d, n, 1, &s);  // T = A x_1 x_1
  f(s, dt);
  f(shape2(n[0], prod_range(n, 2, d), 1), vdt);
  make_shape(d, n, 0, &s);  // W_1 = A x_0 x_0
  f(s, dt);
  f(shape2(n[1], prod_range(n, 2, d), 1), vdt);
  for (int j = 2; j < d; j++) {
    f(shape2(n[j - 1], prod_range(n, j, d), 0), vdt);
    if (j < d - 1) f(shape2(n[j], prod_range(n, j + 1, d), 1), vdt);
  }
}

HopmPlan make_hopm_plan(int order, const int64_t* dims, tvc_dtype dt) {
  HopmPlan hp;
  hp.d = order;
  for (int i = 0; i < order; i++) hp.dims[i] = dims[i];
  hp.N = prod_range(dims, 0, order);
  hp.vs = vec_size(dt);
  const int64_t n0 = dims[0], n1 = dims[1];
  const int64_t bufA = std::max(hp.N / n0, hp.N / n1);
  const int64_t bufB = (order >= 3) ? hp.N / (n0 * n1) : 1;
  const int64_t wlen = (order >= 4) ? hp.N / (n0 * n1) : 1;
  int64_t zlen = 1;
  for (int i = 0; i < order; i++) zlen = std::max(zlen, dims[i]);
  size_t tw = 0;
  // Plan every TVC for a 256-byte aligned operand (the workspace and torch
  // buffers are), keeping the largest workspace any of them needs; operands
  // of other alignments only use smaller plans.
  for_each_tvc(hp, dt, [&](const Shape& s, tvc_dtype t) {
    for (uintptr_t al = elem_size(t); al <= 256; al *= 2)
      tw = std::max(tw, tvc_ws_bytes(s, t, reinterpret_cast<const void*>(al)));
  });
  hp.tvc_ws = tw;
  size_t off = 0;
  hp.off_state = off;
  off += align_up(sizeof(HopmState), 256);
  hp.off_bufA = off;
  off += align_up((size_t)bufA * hp.vs, 256);
  hp.off_bufB = off;
  off += align_up((size_t)bufB * hp.vs, 256);
  hp.off_w = off;
  off += align_up((size_t)wlen * hp.vs, 256);
  hp.off_z = off;
  off += align_up((size_t)zlen * hp.vs, 256);
  hp.off_tvc = off;
  off += align_up(tw, 256);
  hp.total = off;
  return hp;
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096)); }

}  // namespace

size_t hopm_ws_bytes(int order, const int64_t* dims, tvc_dtype dt) { return make_hopm_plan(order, dims, dt).total; }

// Queues `iters` sweeps on `stream`.  x[m] are device vectors (FP64 for F64,
// FP32 otherwise), updated in place.
tvc_status hopm_launch(const void* A, int order, const int64_t* dims, void* const* x, int iters, double tol,
                       double* lam_out, int* sweeps_out, int* status_out, double* lam_hist, tvc_dtype dt,
                       const float* scales, void* ws, size_t ws_bytes, cudaStream_t st) {
  const HopmPlan hp = make_hopm_plan(order, dims, dt);
  if (ws == nullptr || ws_bytes < hp.total) return TVC_ERR_WORKSPACE;
  char* w = static_cast<char*>(ws);
  HopmState* state = reinterpret_cast<HopmState*>(w + hp.off_state);
  const int* done = &state->done;
  void* bufA = w + hp.off_bufA;
  void* bufB = w + hp.off_bufB;
  void* wv = w + hp.off_w;
  void* z = w + hp.off_z;
  void* tws = w + hp.off_tvc;
  const int d = order;
  const int64_t* n = dims;
  const tvc_dtype vdt = (dt == TVC_F64) ? TVC_F64 : TVC_F32;
  const bool f64 = (dt == TVC_F64);
  tvc_status rc = TVC_OK;
  int launches = 0;
  auto tvc2 = [&](const void* X, int64_t a, int64_t b, int mode, const void* xv, void* y, tvc_dtype t,
                  const float* sc) {
    if (rc != TVC_OK) return;
    rc = tvc_launch(X, shape2(a, b, mode), xv, y, t, sc, 1.0, 0.0, tws, hp.tvc_ws, st, done);
  };
  auto tvcd = [&](int mode, const void* xv, void* y) {
    if (rc != TVC_OK) return;
    Shape s;
    make_shape(d, n, mode, &s);
    rc = tvc_launch(A, s, xv, y, dt, scales, 1.0, 0.0, tws, hp.tvc_ws, st, done);
  };
  auto outer = [&](int from) {  // w = x_from (x) ... (x) x_{d-1}
    OuterArgs oa{};
    oa.nm = d - from;
    for (int m = from; m < d; m++) {
      oa.dims[m - from] = n[m];
      oa.xs[m - from] = x[m];
    }
    const int64_t len = prod_range(n, from, d);
    if (f64)
      hopm_outer_kernel<double><<<grid_for(len), 256, 0, st>>>(static_cast<double*>(wv), len, oa, state);
    else
      hopm_outer_kernel<float><<<grid_for(len), 256, 0, st>>>(static_cast<float*>(wv), len, oa, state);
    launches++;
  };
  auto normalize = [&](const void* zz, int j) {
    const int last = (j == d - 1);
    if (f64)
      hopm_normalize_kernel<double><<<1, kNormThreads, 0, st>>>(static_cast<const double*>(zz), static_cast<double*>(x[j]),
                                                                n[j], last, tol, state, lam_out, sweeps_out, status_out,
                                                                lam_hist);
    else
      hopm_normalize_kernel<float><<<1, kNormThreads, 0, st>>>(static_cast<const float*>(zz), static_cast<float*>(x[j]),
                                                               n[j], last, tol, state, lam_out, sweeps_out, status_out,
                                                               lam_hist);
    launches++;
  };
  hopm_init_kernel<<<1, 1, 0, st>>>(state);
  launches++;
  for (int it = 0; it < iters && rc == TVC_OK; it++) {
    if (d == 2) {
      tvcd(1, x[1], z);
      normalize(z, 0);
      tvcd(0, x[0], z);
      normalize(z, 1);
      continue;
    }
    const int64_t rest2 = prod_range(n, 2, d);
    // j = 0
    tvcd(1, x[1], bufA);
    if (d == 3) {
      tvc2(bufA, n[0], n[2], 1, x[2], z, vdt, nullptr);
    } else {
      outer(2);
      tvc2(bufA, n[0], rest2, 1, wv, z, vdt, nullptr);
    }
    normalize(z, 0);
    // j = 1
    tvcd(0, x[0], bufA);
    if (d == 3) {
      tvc2(bufA, n[1], n[2], 1, x[2], z, vdt, nullptr);
    } else {
      outer(2);
      tvc2(bufA, n[1], rest2, 1, wv, z, vdt, nullptr);
    }
    normalize(z, 1);
    // j >= 2
    void* prev = bufA;
    void* next = bufB;
    for (int j = 2; j < d && rc == TVC_OK; j++) {
      tvc2(prev, n[j - 1], prod_range(n, j, d), 0, x[j - 1], next, vdt, nullptr);
      if (j == d - 1) {
        normalize(next, j);
      } else {
        if (j == d - 2) {
          tvc2(next, n[j], n[d - 1], 1, x[d - 1], z, vdt, nullptr);
        } else {
          outer(j + 1);
          tvc2(next, n[j], prod_range(n, j + 1, d), 1, wv, z, vdt, nullptr);
        }
        normalize(z, j);
      }
      std::swap(prev, next);
    }
  }
  count_launches(launches);
  if (rc != TVC_OK) return rc;
  return cuda_status(cudaGetLastError());
}

}  // namespace tvcg

using namespace tvcg;

extern "C" size_t hopm_workspace_size(int order, const int64_t* dims, tvc_dtype dtype) {
  if (!valid_dtype(dtype) || order < 2 || check_dims(order, dims, nullptr) != TVC_OK) return 0;
  return hopm_ws_bytes(order, dims, dtype);
}

extern "C" tvc_status hopm(const void* A, int order, const int64_t* dims, void* const* x, int iters, double tol,
                           double* lambda_out, int* sweeps_out, int* status_out, double* lambda_hist,
                           tvc_dtype dtype, const float* slab_scales, void* workspace, size_t ws_bytes,
                           tvc_stream_t stream) {
  if (!valid_dtype(dtype) || order < 2 || !A || !x || iters < 0 || !(tol >= 0.0)) return TVC_ERR_INVALID_ARG;
  if (check_dims(order, dims, nullptr) != TVC_OK) return TVC_ERR_INVALID_ARG;
  const size_t vs = vec_size(dtype);
  if (!aligned(A, elem_size(dtype))) return TVC_ERR_INVALID_ARG;
  for (int m = 0; m < order; m++)
    if (!x[m] || !aligned(x[m], vs)) return TVC_ERR_INVALID_ARG;
  return hopm_launch(A, order, dims, x, iters, tol, lambda_out, sweeps_out, status_out, lambda_hist, dtype,
                     slab_scales, workspace, ws_bytes, (cudaStream_t)stream);
}
