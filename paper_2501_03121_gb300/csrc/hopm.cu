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
#include <vector>

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
  const float* scale0;  // nullable: the first factor times scale0[its index] (slab scales)
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
    if (oa.scale0) acc *= (V)oa.scale0[dig[0]];
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
                                                                     int* status_out, double* lam_hist,
                                                                     double* sigma_cap) {
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
    if (sigma_cap) *sigma_cap = sigma;
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

// --------------------------------------------------- backward kernels ----

// Adjoint of the normalisation x = z/||z|| (sigma = ||z||):
//   gz = (g - x <x, g>) / sigma + g_sigma x
// with <x, g> in FP64 (fixed-order block reduction).  g_sigma (nullable) is
// the upstream gradient of lambda, used for the last update only.
template <class V>
__global__ void __launch_bounds__(kNormThreads) hopm_bw_gz_kernel(const V* __restrict__ x, const V* __restrict__ g,
                                                                 const double* sigma, const double* gsig, int64_t n,
                                                                 V* __restrict__ gz) {
  __shared__ double red[kNormThreads];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kNormThreads) s = fma((double)x[i], (double)g[i], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = kNormThreads / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  const double dot = red[0];
  const double inv = 1.0 / *sigma;
  const double gs = gsig ? *gsig : 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kNormThreads) {
    const double xi = (double)x[i];
    gz[i] = (V)(((double)g[i] - xi * dot) * inv + gs * xi);
  }
}

template <class V>
__global__ void hopm_axpy_kernel(V* __restrict__ y, const V* __restrict__ x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}

// gA += sum_r prod_m F[r][m][i_m]  (R rank-1 terms of order d, row-major).
constexpr int kCpMaxR = 16;
struct CpArgs {
  int d, R;
  int64_t dims[TVC_MAX_ORDER];
  const void* f[kCpMaxR][TVC_MAX_ORDER];
};

template <class V>
__global__ void __launch_bounds__(256) hopm_cp_kernel(V* __restrict__ gA, int64_t rows, CpArgs ca) {
  // A block handles RB rows (all leading indices but the last mode) per
  // iteration; thread t covers row t / nl, position t % nl of the last mode.
  const int64_t nl = ca.dims[ca.d - 1];
  const int RB = nl >= 256 ? 1 : (int)(256 / nl);
  __shared__ double P[256][kCpMaxR];
  for (int64_t r0 = (int64_t)blockIdx.x * RB; r0 < rows; r0 += (int64_t)gridDim.x * RB) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < RB * ca.R; idx += 256) {
      const int rb = idx / ca.R, r = idx % ca.R;
      const int64_t row = r0 + rb;
      double pr = 0.0;
      if (row < rows) {
        int64_t rem = row;
        pr = 1.0;
        for (int m = ca.d - 2; m >= 0; m--) {
          const int64_t im = rem % ca.dims[m];
          rem /= ca.dims[m];
          pr *= (double)static_cast<const V*>(ca.f[r][m])[im];
        }
      }
      P[rb][r] = pr;
    }
    __syncthreads();
    const int rb = (nl >= 256) ? 0 : (int)(threadIdx.x / nl);
    if (rb >= RB) continue;
    const int64_t row = r0 + rb;
    if (row >= rows) continue;
    for (int64_t k = (nl >= 256) ? threadIdx.x : threadIdx.x % nl; k < nl; k += (nl >= 256) ? 256 : nl) {
      double acc = 0.0;
      for (int r = 0; r < ca.R; r++) acc = fma(P[rb][r], (double)static_cast<const V*>(ca.f[r][ca.d - 1])[k], acc);
      V* p = gA + row * nl + k;
      *p = (V)((double)*p + acc);
    }
  }
}

// ---------------------------------------------------------------- host ----

namespace {

int64_t prod_range(const int64_t* dims, int lo, int hi) {
  int64_t p = 1;
  for (int i = lo; i < hi; i++) p *= dims[i];
  return p;
}

Shape shape2(int64_t a, int64_t b, int mode) {
  Shape s;
  const int64_t d2[2] = {a, b};
  make_shape(2, d2, mode, &s);
  return s;
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096)); }

// Launch context of one power-method run.  In "dry" mode nothing is
// launched: the calls only record the largest TVC workspace they would use,
// which is how the workspace size is computed (the same code path sizes and
// runs).
struct Ctx {
  bool dry = true;
  const void* A = nullptr;
  int d = 0;
  int64_t n[TVC_MAX_ORDER] = {};
  int64_t N = 0;
  tvc_dtype dt = TVC_F64, vdt = TVC_F64;
  const float* scales = nullptr;
  cudaStream_t st = nullptr;
  HopmState* state = nullptr;
  const int* done = nullptr;
  void *bufA = nullptr, *bufB = nullptr, *wv = nullptr, *z = nullptr, *tws = nullptr;
  size_t tws_bytes = 0;
  size_t tvc_need = 0;
  tvc_status rc = TVC_OK;
  int launches = 0;
  void* wchain = nullptr;  // W_j of the running sweep
  void* wother = nullptr;

  bool f64() const { return vdt == TVC_F64; }  // FP64 vectors (TVC_F64, TVC_F32D)

  void tvc(const void* X, const Shape& s, const void* xv, void* y, tvc_dtype t, const float* sc, double beta = 0.0) {
    if (rc != TVC_OK) return;
    if (dry) {
      for (uintptr_t al = elem_size(t); al <= 256; al *= 2)
        tvc_need = std::max(tvc_need, tvc_ws_bytes(s, t, reinterpret_cast<const void*>(al)));
      return;
    }
    rc = tvc_launch(X, s, xv, y, t, sc, 1.0, beta, tws, tws_bytes, st, done);
  }
  void tvcA(int mode, const void* xv, void* y) {
    Shape s;
    make_shape(d, n, mode, &s);
    tvc(A, s, xv, y, dt, scales);
  }
  void outer(int from, void* const* xs) {  // wv = x_from (x) ... (x) x_{d-1}
    if (dry || rc != TVC_OK) return;
    OuterArgs oa{};
    oa.nm = d - from;
    for (int m = from; m < d; m++) {
      oa.dims[m - from] = n[m];
      oa.xs[m - from] = xs[m];
    }
    const int64_t len = prod_range(n, from, d);
    if (f64())
      hopm_outer_kernel<double><<<grid_for(len), 256, 0, st>>>(static_cast<double*>(wv), len, oa, state);
    else
      hopm_outer_kernel<float><<<grid_for(len), 256, 0, st>>>(static_cast<float*>(wv), len, oa, state);
    launches++;
  }
  // z_j = A x_{m != j} x_m with the current vectors xs; updates j of one
  // sweep must come in order 0..d-1 (the W chain).  Returns the buffer of z_j.
  void* z_for(int j, void* const* xs) {
    if (d == 2) {
      tvcA(1 - j, xs[1 - j], z);
      return z;
    }
    if (j == 0 || j == 1) {
      void* T = bufA;
      tvcA(j == 0 ? 1 : 0, xs[j == 0 ? 1 : 0], T);
      const int64_t rest2 = prod_range(n, 2, d);
      if (d == 3) {
        tvc(T, shape2(n[j], n[2], 1), xs[2], z, vdt, nullptr);
      } else {
        outer(2, xs);
        tvc(T, shape2(n[j], rest2, 1), wv, z, vdt, nullptr);
      }
      wchain = bufA;
      wother = bufB;
      return z;
    }
    void* next = wother;
    tvc(wchain, shape2(n[j - 1], prod_range(n, j, d), 0), xs[j - 1], next, vdt, nullptr);
    wother = wchain;
    wchain = next;
    if (j == d - 1) return next;
    if (j == d - 2) {
      tvc(next, shape2(n[j], n[d - 1], 1), xs[d - 1], z, vdt, nullptr);
    } else {
      outer(j + 1, xs);
      tvc(next, shape2(n[j], prod_range(n, j + 1, d), 1), wv, z, vdt, nullptr);
    }
    return z;
  }
  void normalize(const void* zz, int j, void* xj, double tol, double* lam_out, int* sweeps_out, int* status_out,
                 double* lam_hist, double* sigma_cap) {
    if (dry || rc != TVC_OK) return;
    const int last = (j == d - 1);
    if (f64())
      hopm_normalize_kernel<double><<<1, kNormThreads, 0, st>>>(static_cast<const double*>(zz), static_cast<double*>(xj),
                                                                n[j], last, tol, state, lam_out, sweeps_out, status_out,
                                                                lam_hist, sigma_cap);
    else
      hopm_normalize_kernel<float><<<1, kNormThreads, 0, st>>>(static_cast<const float*>(zz), static_cast<float*>(xj),
                                                               n[j], last, tol, state, lam_out, sweeps_out, status_out,
                                                               lam_hist, sigma_cap);
    launches++;
  }
  void init_state() {
    if (dry) return;
    hopm_init_kernel<<<1, 1, 0, st>>>(state);
    launches++;
  }
  // One Gauss-Seidel sweep on the vectors xs (updated in place).
  void sweep(void* const* xs, double tol, double* lam_out, int* sweeps_out, int* status_out, double* lam_hist,
             double* sigma_cap) {
    for (int j = 0; j < d && rc == TVC_OK; j++) {
      void* zz = z_for(j, xs);
      normalize(zz, j, xs[j], tol, lam_out, sweeps_out, status_out, lam_hist, sigma_cap ? sigma_cap + j : nullptr);
    }
  }
};

// Workspace layout of a forward run.
struct FwdLayout {
  size_t off_state = 0, off_bufA = 0, off_bufB = 0, off_w = 0, off_z = 0, off_tvc = 0, total = 0, tvc = 0;
};

FwdLayout fwd_layout(int order, const int64_t* dims, tvc_dtype dt, size_t base) {
  FwdLayout L;
  const size_t vs = vec_size(dt);
  const int64_t N = prod_range(dims, 0, order);
  const int64_t n0 = dims[0], n1 = dims[1];
  const int64_t bufA = std::max(N / n0, N / n1);
  const int64_t bufB = (order >= 3) ? N / (n0 * n1) : 1;
  const int64_t wlen = (order >= 4) ? N / (n0 * n1) : 1;
  int64_t zlen = 1;
  for (int i = 0; i < order; i++) zlen = std::max(zlen, dims[i]);
  Ctx c;
  c.dry = true;
  c.d = order;
  for (int i = 0; i < order; i++) c.n[i] = dims[i];
  c.dt = dt;
  c.vdt = (dt == TVC_F64 || dt == TVC_F32D) ? TVC_F64 : TVC_F32;
  void* dummy[TVC_MAX_ORDER] = {};
  c.sweep(dummy, 0.0, nullptr, nullptr, nullptr, nullptr, nullptr);
  size_t off = base;
  L.off_state = off;
  off += align_up(sizeof(HopmState), 256);
  L.off_bufA = off;
  off += align_up((size_t)bufA * vs, 256);
  L.off_bufB = off;
  off += align_up((size_t)bufB * vs, 256);
  L.off_w = off;
  off += align_up((size_t)wlen * vs, 256);
  L.off_z = off;
  off += align_up((size_t)zlen * vs, 256);
  L.off_tvc = off;
  L.tvc = c.tvc_need;
  off += align_up(c.tvc_need, 256);
  L.total = off;
  return L;
}

void bind(Ctx& c, const FwdLayout& L, void* ws, const void* A, int order, const int64_t* dims, tvc_dtype dt,
          const float* scales, cudaStream_t st) {
  char* w = static_cast<char*>(ws);
  c.dry = false;
  c.A = A;
  c.d = order;
  for (int i = 0; i < order; i++) c.n[i] = dims[i];
  c.N = prod_range(dims, 0, order);
  c.dt = dt;
  c.vdt = (dt == TVC_F64 || dt == TVC_F32D) ? TVC_F64 : TVC_F32;
  c.scales = scales;
  c.st = st;
  c.state = reinterpret_cast<HopmState*>(w + L.off_state);
  c.done = &c.state->done;
  c.bufA = w + L.off_bufA;
  c.bufB = w + L.off_bufB;
  c.wv = w + L.off_w;
  c.z = w + L.off_z;
  c.tws = w + L.off_tvc;
  c.tws_bytes = L.tvc;
}

}  // namespace

size_t hopm_ws_bytes(int order, const int64_t* dims, tvc_dtype dt) { return fwd_layout(order, dims, dt, 0).total; }

// Queues `iters` sweeps on `stream`.  x[m] are device vectors (FP64 for F64,
// FP32 otherwise), updated in place.
tvc_status hopm_launch(const void* A, int order, const int64_t* dims, void* const* x, int iters, double tol,
                       double* lam_out, int* sweeps_out, int* status_out, double* lam_hist, tvc_dtype dt,
                       const float* scales, void* ws, size_t ws_bytes, cudaStream_t st) {
  const FwdLayout L = fwd_layout(order, dims, dt, 0);
  if (ws == nullptr || ws_bytes < L.total) return TVC_ERR_WORKSPACE;
  Ctx c;
  bind(c, L, ws, A, order, dims, dt, scales, st);
  c.init_state();
  for (int it = 0; it < iters && c.rc == TVC_OK; it++) c.sweep(x, tol, lam_out, sweeps_out, status_out, lam_hist, nullptr);
  count_launches(c.launches);
  if (c.rc != TVC_OK) return c.rc;
  return cuda_status(cudaGetLastError());
}

// ------------------------------------------- distributed (virtual ranks)

namespace {

// Workspace of dHOPM_3 over virtual ranks: the shared state and the
// combined vector z, then one forward layout per rank (its W cache,
// intermediate buffers and TVC workspace).
struct DLayout {
  size_t off_state = 0, off_zsum = 0, total = 0;
  std::vector<FwdLayout> rank;
};

DLayout dhopm_layout(int parts, const int64_t* starts, int order, const int64_t* dims, int s, tvc_dtype dt) {
  DLayout D;
  int64_t zlen = 1;
  for (int i = 0; i < order; i++) zlen = std::max(zlen, dims[i]);
  size_t off = 0;
  D.off_state = off;
  off += align_up(sizeof(HopmState), 256);
  D.off_zsum = off;
  off += align_up((size_t)zlen * vec_size(dt), 256);
  int64_t dr[TVC_MAX_ORDER];
  for (int r = 0; r < parts; r++) {
    slab_dims(order, dims, s, starts, r, dr);
    D.rank.push_back(fwd_layout(order, dr, dt, off));
    off = D.rank.back().total;
  }
  D.total = off;
  return D;
}

}  // namespace

size_t dhopm_ws_bytes(int parts, const int64_t* starts, int order, const int64_t* dims, int s, tvc_dtype dt) {
  return dhopm_layout(parts, starts, order, dims, s, dt).total;
}

// Algorithm 1 over `parts` virtual ranks: for each external iteration j,
// every rank runs its local chain (its own W_j, x_s cut to its range), then
// the n_j-entry results are summed over ranks (j != s) or gathered (j = s),
// and the global x_j is normalised once.  All queued on one stream.
tvc_status dhopm_launch(const void* const* slabs, int parts, const int64_t* starts, int order, const int64_t* dims,
                        int s, void* const* x, int iters, double tol, double* lam_out, int* sweeps_out,
                        int* status_out, double* lam_hist, tvc_dtype dt, const float* scales, void* ws,
                        size_t ws_bytes, cudaStream_t st) {
  const DLayout D = dhopm_layout(parts, starts, order, dims, s, dt);
  if (ws == nullptr || ws_bytes < D.total) return TVC_ERR_WORKSPACE;
  char* w = static_cast<char*>(ws);
  const size_t vs = vec_size(dt);
  Ctx g;  // global view: the state, the normalisation of the combined z
  g.dry = false;
  g.d = order;
  for (int i = 0; i < order; i++) g.n[i] = dims[i];
  g.dt = dt;
  g.vdt = (dt == TVC_F64 || dt == TVC_F32D) ? TVC_F64 : TVC_F32;
  g.st = st;
  g.state = reinterpret_cast<HopmState*>(w + D.off_state);
  g.done = &g.state->done;
  void* zsum = w + D.off_zsum;
  std::vector<Ctx> c(parts);
  std::vector<std::vector<void*>> xr(parts, std::vector<void*>(order));
  int64_t dr[TVC_MAX_ORDER];
  for (int r = 0; r < parts; r++) {
    slab_dims(order, dims, s, starts, r, dr);
    const float* sc = scales ? scales + (s == 0 ? starts[r] : 0) : nullptr;
    bind(c[r], D.rank[r], ws, slabs[r], order, dr, dt, sc, st);
    c[r].state = g.state;  // one state: the done flag stops every rank
    c[r].done = g.done;
    for (int m = 0; m < order; m++)
      xr[r][m] = (m == s) ? static_cast<void*>(static_cast<char*>(x[m]) + (size_t)starts[r] * vs) : x[m];
  }
  g.init_state();
  tvc_status rc = TVC_OK;
  int combines = 0;
  const void* zp[TVC_MAX_PARTS];
  for (int it = 0; it < iters && rc == TVC_OK; it++) {
    for (int j = 0; j < order && rc == TVC_OK; j++) {
      for (int r = 0; r < parts; r++) {
        zp[r] = c[r].z_for(j, xr[r].data());
        if (c[r].rc != TVC_OK) rc = c[r].rc;
      }
      if (rc != TVC_OK) break;
      // j != s: array reduction; j == s: array gather (Algorithm 1).
      rc = combine_parts(zp, parts, starts, dims[j], zsum, g.vdt, j == s ? 1 : 0, 1.0, 0.0, st, g.done);
      combines++;
      g.normalize(zsum, j, x[j], tol, lam_out, sweeps_out, status_out, lam_hist, nullptr);
    }
  }
  int launches = g.launches;
  for (int r = 0; r < parts; r++) launches += c[r].launches;
  count_launches(launches);
  (void)combines;  // counted by combine_parts
  if (rc != TVC_OK) return rc;
  return cuda_status(cudaGetLastError());
}

// ------------------------------------------------------------ Jacobi

namespace {

// Jacobi HOPM (not the paper's Algorithm 1): every z_j of a sweep from the
// previous sweep's vectors.  With C = n_{d-1} and R = N / C:
//   w       = x_0 (x) ... (x) x_{d-2}           (R entries; slab scales of
//                                                narrow storage folded in)
//   T       = A x_{d-1} x_{d-1}                 (R entries)
//   z_{d-1} = A^T w over the R x C view          (C entries)
//   z_j     = T contracted with x_m, m != j, m < d-1   (j < d-1; T is small)
// then every x_j <- z_j / ||z_j||, lambda = ||z_{d-1}|| (FP64 norms).
struct JacobiCtx {
  bool dry = true;
  const void* A = nullptr;
  int d = 0;
  int64_t n[TVC_MAX_ORDER] = {};
  int64_t R = 0, C = 0;
  tvc_dtype dt = TVC_F64, vdt = TVC_F64;
  const float* scales = nullptr;
  cudaStream_t st = nullptr;
  HopmState* state = nullptr;
  void *T = nullptr, *T1 = nullptr, *wv = nullptr, *tws = nullptr;
  void* z[TVC_MAX_ORDER] = {};
  size_t tws_bytes = 0, tvc_need = 0;
  tvc_status rc = TVC_OK;
  int launches = 0;

  bool f64() const { return vdt == TVC_F64; }
  void tvc(const void* X, const Shape& s, const void* xv, void* y, tvc_dtype t, const float* sc) {
    if (rc != TVC_OK) return;
    if (dry) {
      for (uintptr_t al = elem_size(t); al <= 256; al *= 2)
        tvc_need = std::max(tvc_need, tvc_ws_bytes(s, t, reinterpret_cast<const void*>(al)));
      return;
    }
    rc = tvc_launch(X, s, xv, y, t, sc, 1.0, 0.0, tws, tws_bytes, st, &state->done);
  }
  // out = x_lo (x) ... (x) x_{hi-1} (the first factor times scale0 when given)
  void outer(int lo, int hi, void* const* xs, void* out, const float* scale0) {
    if (dry || rc != TVC_OK) return;
    OuterArgs oa{};
    oa.nm = hi - lo;
    for (int m = lo; m < hi; m++) {
      oa.dims[m - lo] = n[m];
      oa.xs[m - lo] = xs[m];
    }
    oa.scale0 = scale0;
    const int64_t len = prod_range(n, lo, hi);
    if (f64())
      hopm_outer_kernel<double><<<grid_for(len), 256, 0, st>>>(static_cast<double*>(out), len, oa, state);
    else
      hopm_outer_kernel<float><<<grid_for(len), 256, 0, st>>>(static_cast<float*>(out), len, oa, state);
    launches++;
  }
  void normalize(int j, void* xj, double tol, double* lam_out, int* sweeps_out, int* status_out, double* lam_hist) {
    if (dry || rc != TVC_OK) return;
    const int last = (j == d - 1);
    if (f64())
      hopm_normalize_kernel<double><<<1, kNormThreads, 0, st>>>(static_cast<const double*>(z[j]), static_cast<double*>(xj),
                                                                n[j], last, tol, state, lam_out, sweeps_out, status_out,
                                                                lam_hist, nullptr);
    else
      hopm_normalize_kernel<float><<<1, kNormThreads, 0, st>>>(static_cast<const float*>(z[j]), static_cast<float*>(xj),
                                                               n[j], last, tol, state, lam_out, sweeps_out, status_out,
                                                               lam_hist, nullptr);
    launches++;
  }
  void sweep(void* const* xs, double tol, double* lam_out, int* sweeps_out, int* status_out, double* lam_hist) {
    const bool narrow = (dt == TVC_BF16 || dt == TVC_E4M3 || dt == TVC_F16) && scales != nullptr;
    // w (slab scales folded into the x_0 factor), then the two views of A
    const void* w = xs[0];
    if (d > 2 || narrow) {
      outer(0, d - 1, xs, wv, narrow ? scales : nullptr);
      w = wv;
    }
    if (dual_supported(R, C, dt, dry ? reinterpret_cast<const void*>(256) : A)) {
      // both products from ONE pass over A (FP32 / BF16 / F16 / E4M3)
      if (dry) {
        tvc_need = std::max(tvc_need, dual_ws_bytes(R, C, dt, nullptr));
      } else if (rc == TVC_OK) {
        rc = dual_launch(A, R, C, dt, static_cast<const float*>(xs[d - 1]), static_cast<const float*>(w),
                         narrow ? scales : nullptr, R / n[0], static_cast<float*>(T), static_cast<float*>(z[d - 1]),
                         tws, tws_bytes, st, &state->done);
      }
    } else {
      Shape s;
      make_shape(d, n, d - 1, &s);
      tvc(A, s, xs[d - 1], T, dt, scales);               // T = A x_{d-1} x_{d-1}
      tvc(A, shape2(R, C, 0), w, z[d - 1], dt, nullptr);  // z_{d-1} = A^T w
    }
    // z_j, j < d-1, from T (order d-1: n_0 .. n_{d-2}): contract the modes
    // after j, then those before j, each group against its outer product
    // (modes of size one included: their x entry is a factor too)
    for (int j = 0; j < d - 1 && rc == TVC_OK; j++) {
      const int64_t u = prod_range(n, 0, j), v = prod_range(n, j + 1, d - 1);
      const bool has_pre = j > 0, has_post = j + 1 < d - 1;
      const void* src = T;
      if (has_post) {
        outer(j + 1, d - 1, xs, wv, nullptr);
        void* dst = has_pre ? T1 : z[j];
        tvc(T, shape2(u * n[j], v, 1), wv, dst, vdt, nullptr);
        src = dst;
      }
      if (has_pre) {
        outer(0, j, xs, wv, nullptr);
        tvc(src, shape2(u, n[j], 0), wv, z[j], vdt, nullptr);
      }
      // neither: d = 2, where T is z_0 itself (see the launch)
    }
    for (int j = 0; j < d && rc == TVC_OK; j++) normalize(j, xs[j], tol, lam_out, sweeps_out, status_out, lam_hist);
  }
};

struct JLayout {
  size_t off_state = 0, off_T = 0, off_T1 = 0, off_w = 0, off_tvc = 0, total = 0, tvc = 0;
  size_t off_z[TVC_MAX_ORDER] = {};
};

JLayout jacobi_layout(int order, const int64_t* dims, tvc_dtype dt) {
  JLayout L;
  const size_t vs = vec_size(dt);
  const int64_t N = prod_range(dims, 0, order);
  const int64_t R = N / dims[order - 1];
  JacobiCtx c;
  c.dry = true;
  c.d = order;
  for (int i = 0; i < order; i++) c.n[i] = dims[i];
  c.R = R;
  c.C = dims[order - 1];
  c.dt = dt;
  c.vdt = (dt == TVC_F64 || dt == TVC_F32D) ? TVC_F64 : TVC_F32;
  void* dummy[TVC_MAX_ORDER] = {};
  c.sweep(dummy, 0.0, nullptr, nullptr, nullptr, nullptr);
  size_t off = 0;
  L.off_state = off;
  off += align_up(sizeof(HopmState), 256);
  L.off_T = off;
  off += align_up((size_t)R * vs, 256);
  L.off_T1 = off;
  off += align_up((size_t)R * vs, 256);
  L.off_w = off;
  off += align_up((size_t)R * vs, 256);
  for (int j = 0; j < order; j++) {
    L.off_z[j] = off;
    off += align_up((size_t)dims[j] * vs, 256);
  }
  L.off_tvc = off;
  L.tvc = c.tvc_need;
  off += align_up(c.tvc_need, 256);
  L.total = off;
  return L;
}

}  // namespace

size_t hopm_jacobi_ws_bytes(int order, const int64_t* dims, tvc_dtype dt) {
  return jacobi_layout(order, dims, dt).total;
}

tvc_status hopm_jacobi_launch(const void* A, int order, const int64_t* dims, void* const* x, int iters, double tol,
                              double* lam_out, int* sweeps_out, int* status_out, double* lam_hist, tvc_dtype dt,
                              const float* scales, void* ws, size_t ws_bytes, cudaStream_t st) {
  const JLayout L = jacobi_layout(order, dims, dt);
  if (ws == nullptr || ws_bytes < L.total) return TVC_ERR_WORKSPACE;
  char* w = static_cast<char*>(ws);
  JacobiCtx c;
  c.dry = false;
  c.A = A;
  c.d = order;
  for (int i = 0; i < order; i++) c.n[i] = dims[i];
  c.C = dims[order - 1];
  c.R = prod_range(dims, 0, order) / c.C;
  c.dt = dt;
  c.vdt = (dt == TVC_F64 || dt == TVC_F32D) ? TVC_F64 : TVC_F32;
  c.scales = scales;
  c.st = st;
  c.state = reinterpret_cast<HopmState*>(w + L.off_state);
  c.T = w + L.off_T;
  c.T1 = w + L.off_T1;
  c.wv = w + L.off_w;
  for (int j = 0; j < order; j++) c.z[j] = w + L.off_z[j];
  if (order == 2) c.T = c.z[0];  // T = A x_1 x_1 is z_0
  c.tws = w + L.off_tvc;
  c.tws_bytes = L.tvc;
  hopm_init_kernel<<<1, 1, 0, st>>>(c.state);
  c.launches++;
  for (int it = 0; it < iters && c.rc == TVC_OK; it++) c.sweep(x, tol, lam_out, sweeps_out, status_out, lam_hist);
  count_launches(c.launches);
  if (c.rc != TVC_OK) return c.rc;
  return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------- backward

namespace {

// Backward workspace: the forward layout, then
//   ckpt  iters x sum(n) vectors (the vectors at the start of every sweep)
//   xw    sum(n)   working vectors (recomputed iterates of one sweep)
//   gbar  sum(n)   adjoints of the current vectors
//   gzs   sum(n)   adjoints of z_j of one sweep (the rank-1 factors of gA)
//   sig   d doubles (norms of one sweep)
//   W, P0, P1      N / min_j n_j each (A x_j gz and its further contractions)
struct BwdLayout {
  FwdLayout f;
  size_t off_ckpt = 0, off_xw = 0, off_gbar = 0, off_gzs = 0, off_sig = 0, off_W = 0, off_P0 = 0, off_P1 = 0;
  size_t total = 0;
  int64_t sumn = 0, wmax = 0;
};

// Contracts the (d-1)-tensor X (modes `ids`, sizes `sz`) with vecs[k] for
// every mode k other than `keep`, leaving the n_keep-vector; the last
// contraction adds into gout (beta = 1).
void all_but_one(Ctx& c, const void* X, int nd, const int* ids, const int64_t* sz, int keep, void* const* vecs,
                 void* gout, void* P0, void* P1) {
  int cid[TVC_MAX_ORDER];
  int64_t csz[TVC_MAX_ORDER];
  for (int q = 0; q < nd; q++) {
    cid[q] = ids[q];
    csz[q] = sz[q];
  }
  const void* cur = X;
  void* bufs[2] = {P0, P1};
  int nb = 0;
  if (nd == 1) {  // X is already the vector
    if (!c.dry && c.rc == TVC_OK) {
      const int64_t len = csz[0];
      if (c.f64())
        hopm_axpy_kernel<double><<<grid_for(len), 256, 0, c.st>>>(static_cast<double*>(gout),
                                                                  static_cast<const double*>(cur), len);
      else
        hopm_axpy_kernel<float><<<grid_for(len), 256, 0, c.st>>>(static_cast<float*>(gout),
                                                                 static_cast<const float*>(cur), len);
      c.launches++;
    }
    return;
  }
  while (nd > 1) {
    int p = (cid[0] != keep) ? 0 : 1;  // first mode that is not kept
    Shape s;
    make_shape(nd, csz, p, &s);
    const bool last = (nd == 2);
    void* out = last ? gout : bufs[nb];
    c.tvc(cur, s, vecs[cid[p]], out, c.vdt, nullptr, last ? 1.0 : 0.0);
    for (int q = p; q < nd - 1; q++) {
      cid[q] = cid[q + 1];
      csz[q] = csz[q + 1];
    }
    nd--;
    cur = out;
    nb ^= 1;
  }
}

BwdLayout bwd_layout(int order, const int64_t* dims, tvc_dtype dt, int iters) {
  BwdLayout L;
  L.f = fwd_layout(order, dims, dt, 0);
  const size_t vs = vec_size(dt);
  int64_t sumn = 0, nmin = dims[0];
  for (int i = 0; i < order; i++) {
    sumn += dims[i];
    nmin = std::min(nmin, dims[i]);
  }
  const int64_t N = prod_range(dims, 0, order);
  L.sumn = sumn;
  L.wmax = N / nmin;
  // Size the TVCs of the reverse pass with a dry run of it.
  Ctx c;
  c.dry = true;
  c.d = order;
  for (int i = 0; i < order; i++) c.n[i] = dims[i];
  c.dt = dt;
  c.vdt = (dt == TVC_F64 || dt == TVC_F32D) ? TVC_F64 : TVC_F32;
  void* dummy[TVC_MAX_ORDER] = {};
  for (int j = 0; j < order; j++) {
    c.tvcA(j, nullptr, nullptr);
    int ids[TVC_MAX_ORDER];
    int64_t sz[TVC_MAX_ORDER];
    int nd = 0;
    for (int m = 0; m < order; m++)
      if (m != j) {
        ids[nd] = m;
        sz[nd] = dims[m];
        nd++;
      }
    for (int m = 0; m < order; m++)
      if (m != j) all_but_one(c, nullptr, nd, ids, sz, m, dummy, nullptr, nullptr, nullptr);
  }
  size_t off = L.f.total;
  // The forward's TVC region must hold the reverse pass's TVCs too.
  const size_t extra_tvc = c.tvc_need > L.f.tvc ? align_up(c.tvc_need - L.f.tvc, 256) : 0;
  L.f.tvc = std::max(L.f.tvc, c.tvc_need);
  off += extra_tvc;
  L.off_ckpt = off;
  off += align_up((size_t)iters * sumn * vs, 256);
  L.off_xw = off;
  off += align_up((size_t)sumn * vs, 256);
  L.off_gbar = off;
  off += align_up((size_t)sumn * vs, 256);
  L.off_gzs = off;
  off += align_up((size_t)sumn * vs, 256);
  L.off_sig = off;
  off += align_up((size_t)order * 8, 256);
  L.off_W = off;
  off += align_up((size_t)L.wmax * vs, 256);
  L.off_P0 = off;
  off += align_up((size_t)L.wmax * vs, 256);
  L.off_P1 = off;
  off += align_up((size_t)L.wmax * vs, 256);
  L.total = off;
  return L;
}

}  // namespace

// Reverse-mode gradient of a fixed-count power method (iters sweeps, no
// early stop) with respect to A and to the start vectors, given upstream
// gradients of the final vectors (gx_final[m], nullable) and of lambda
// (g_lambda, device double, nullable).  Per sweep (last to first): the
// sweep is recomputed from its checkpoint, then the updates are reversed:
//   gz  = normalisation adjoint of x_j = z_j/||z_j||
//   gA += gz (at mode j) (x) the other vectors as they were at the update
//   W   = A x_j gz;  gbar_m += W contracted with the other vectors, m != j
//   gbar_j = 0 (x_j's old value was overwritten)
// gA is written (not accumulated); gstart[m] (nullable) receive gbar_m.
tvc_status hopm_backward_launch(const void* A, int order, const int64_t* dims, void* const* x0, int iters,
                                void* const* gx_final, const double* g_lambda, void* gA, void* const* gstart,
                                tvc_dtype dt, const float* scales, void* ws, size_t ws_bytes, cudaStream_t st) {
  const BwdLayout L = bwd_layout(order, dims, dt, iters);
  if (ws == nullptr || ws_bytes < L.total) return TVC_ERR_WORKSPACE;
  const size_t vs = vec_size(dt);
  char* w = static_cast<char*>(ws);
  Ctx c;
  bind(c, L.f, ws, A, order, dims, dt, scales, st);
  const int d = order;
  int64_t off[TVC_MAX_ORDER + 1];
  off[0] = 0;
  for (int m = 0; m < d; m++) off[m + 1] = off[m] + dims[m];
  auto vec_at = [&](size_t base, int m) -> void* { return w + base + (size_t)off[m] * vs; };
  void* xw[TVC_MAX_ORDER];
  void* gbar[TVC_MAX_ORDER];
  void* gzs[TVC_MAX_ORDER];
  for (int m = 0; m < d; m++) {
    xw[m] = vec_at(L.off_xw, m);
    gbar[m] = vec_at(L.off_gbar, m);
    gzs[m] = vec_at(L.off_gzs, m);
  }
  auto ckpt = [&](int t, int m) -> void* { return w + L.off_ckpt + ((size_t)t * L.sumn + off[m]) * vs; };
  double* sig = reinterpret_cast<double*>(w + L.off_sig);
  void* W = w + L.off_W;
  void* P0 = w + L.off_P0;
  void* P1 = w + L.off_P1;
  const int64_t N = prod_range(dims, 0, d);
  // 1. forward with checkpoints
  c.init_state();
  for (int m = 0; m < d; m++) cudaMemcpyAsync(xw[m], x0[m], dims[m] * vs, cudaMemcpyDeviceToDevice, st);
  for (int t = 0; t < iters && c.rc == TVC_OK; t++) {
    for (int m = 0; m < d; m++) cudaMemcpyAsync(ckpt(t, m), xw[m], dims[m] * vs, cudaMemcpyDeviceToDevice, st);
    c.sweep(xw, 0.0, nullptr, nullptr, nullptr, nullptr, nullptr);
  }
  // 2. adjoints of the final vectors
  for (int m = 0; m < d; m++) {
    if (gx_final && gx_final[m])
      cudaMemcpyAsync(gbar[m], gx_final[m], dims[m] * vs, cudaMemcpyDeviceToDevice, st);
    else
      cudaMemsetAsync(gbar[m], 0, dims[m] * vs, st);
  }
  cudaMemsetAsync(gA, 0, (size_t)N * vs, st);
  // 3. reverse over sweeps
  for (int t = iters - 1; t >= 0 && c.rc == TVC_OK; t--) {
    for (int m = 0; m < d; m++) cudaMemcpyAsync(xw[m], ckpt(t, m), dims[m] * vs, cudaMemcpyDeviceToDevice, st);
    c.init_state();
    c.sweep(xw, 0.0, nullptr, nullptr, nullptr, nullptr, sig);  // xw now holds the sweep's new vectors
    for (int j = d - 1; j >= 0 && c.rc == TVC_OK; j--) {
      // vectors at the time of update j: new for m < j, old (checkpoint) for m > j
      void* cur[TVC_MAX_ORDER];
      for (int m = 0; m < d; m++) cur[m] = (m < j) ? xw[m] : ckpt(t, m);
      const double* gs = (t == iters - 1 && j == d - 1) ? g_lambda : nullptr;
      if (c.f64())
        hopm_bw_gz_kernel<double><<<1, kNormThreads, 0, st>>>(static_cast<const double*>(xw[j]),
                                                              static_cast<const double*>(gbar[j]), sig + j, gs,
                                                              dims[j], static_cast<double*>(gzs[j]));
      else
        hopm_bw_gz_kernel<float><<<1, kNormThreads, 0, st>>>(static_cast<const float*>(xw[j]),
                                                             static_cast<const float*>(gbar[j]), sig + j, gs, dims[j],
                                                             static_cast<float*>(gzs[j]));
      c.launches++;
      c.tvcA(j, gzs[j], W);
      int ids[TVC_MAX_ORDER];
      int64_t sz[TVC_MAX_ORDER];
      int nd = 0;
      for (int m = 0; m < d; m++)
        if (m != j) {
          ids[nd] = m;
          sz[nd] = dims[m];
          nd++;
        }
      for (int m = 0; m < d; m++)
        if (m != j) all_but_one(c, W, nd, ids, sz, m, cur, gbar[m], P0, P1);
      cudaMemsetAsync(gbar[j], 0, dims[j] * vs, st);
    }
    // gA += sum_j gz_j (x) (the other vectors at update j)
    CpArgs ca{};
    ca.d = d;
    ca.R = d;
    for (int m = 0; m < d; m++) ca.dims[m] = dims[m];
    for (int j = 0; j < d; j++)
      for (int m = 0; m < d; m++) ca.f[j][m] = (m == j) ? gzs[j] : ((m < j) ? xw[m] : ckpt(t, m));
    const int64_t rows = N / dims[d - 1];
    const int64_t RB = dims[d - 1] >= 256 ? 1 : 256 / dims[d - 1];
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((rows + RB - 1) / RB, (int64_t)device_sms() * 8));
    if (c.f64())
      hopm_cp_kernel<double><<<blocks, 256, 0, st>>>(static_cast<double*>(gA), rows, ca);
    else
      hopm_cp_kernel<float><<<blocks, 256, 0, st>>>(static_cast<float*>(gA), rows, ca);
    c.launches++;
  }
  if (gstart)
    for (int m = 0; m < d; m++)
      if (gstart[m]) cudaMemcpyAsync(gstart[m], gbar[m], dims[m] * vs, cudaMemcpyDeviceToDevice, st);
  count_launches(c.launches);
  if (c.rc != TVC_OK) return c.rc;
  return cuda_status(cudaGetLastError());
}

size_t hopm_bwd_ws_bytes(int order, const int64_t* dims, tvc_dtype dt, int iters) {
  return bwd_layout(order, dims, dt, iters).total;
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

extern "C" size_t dhopm_workspace_size(int parts, const int64_t* starts, int order, const int64_t* dims, int s,
                                       tvc_dtype dtype) {
  if (!valid_dtype(dtype) || order < 2 || check_split(parts, starts, order, dims, s) != TVC_OK) return 0;
  return dhopm_ws_bytes(parts, starts, order, dims, s, dtype);
}

extern "C" tvc_status dhopm(const void* const* slabs, int parts, const int64_t* starts, int order,
                            const int64_t* dims, int s, void* const* x, int iters, double tol, double* lambda_out,
                            int* sweeps_out, int* status_out, double* lambda_hist, tvc_dtype dtype,
                            const float* slab_scales, void* workspace, size_t ws_bytes, tvc_stream_t stream) {
  if (!valid_dtype(dtype) || order < 2 || !slabs || !x || iters < 0 || !(tol >= 0.0)) return TVC_ERR_INVALID_ARG;
  if (check_split(parts, starts, order, dims, s) != TVC_OK) return TVC_ERR_INVALID_ARG;
  const size_t vs = vec_size(dtype);
  for (int r = 0; r < parts; r++)
    if (!slabs[r] || !aligned(slabs[r], elem_size(dtype))) return TVC_ERR_INVALID_ARG;
  for (int m = 0; m < order; m++)
    if (!x[m] || !aligned(x[m], vs)) return TVC_ERR_INVALID_ARG;
  return dhopm_launch(slabs, parts, starts, order, dims, s, x, iters, tol, lambda_out, sweeps_out, status_out,
                      lambda_hist, dtype, slab_scales, workspace, ws_bytes, (cudaStream_t)stream);
}

extern "C" size_t hopm_jacobi_workspace_size(int order, const int64_t* dims, tvc_dtype dtype) {
  if (!valid_dtype(dtype) || order < 2 || check_dims(order, dims, nullptr) != TVC_OK) return 0;
  return hopm_jacobi_ws_bytes(order, dims, dtype);
}

extern "C" tvc_status hopm_jacobi(const void* A, int order, const int64_t* dims, void* const* x, int iters, double tol,
                                  double* lambda_out, int* sweeps_out, int* status_out, double* lambda_hist,
                                  tvc_dtype dtype, const float* slab_scales, void* workspace, size_t ws_bytes,
                                  tvc_stream_t stream) {
  if (!valid_dtype(dtype) || order < 2 || !A || !x || iters < 0 || !(tol >= 0.0)) return TVC_ERR_INVALID_ARG;
  if (check_dims(order, dims, nullptr) != TVC_OK) return TVC_ERR_INVALID_ARG;
  const size_t vs = vec_size(dtype);
  if (!aligned(A, elem_size(dtype))) return TVC_ERR_INVALID_ARG;
  for (int m = 0; m < order; m++)
    if (!x[m] || !aligned(x[m], vs)) return TVC_ERR_INVALID_ARG;
  return hopm_jacobi_launch(A, order, dims, x, iters, tol, lambda_out, sweeps_out, status_out, lambda_hist, dtype,
                            slab_scales, workspace, ws_bytes, (cudaStream_t)stream);
}

extern "C" size_t hopm_backward_workspace_size(int order, const int64_t* dims, tvc_dtype dtype, int iters) {
  if (!valid_dtype(dtype) || order < 2 || iters < 0 || check_dims(order, dims, nullptr) != TVC_OK) return 0;
  return hopm_bwd_ws_bytes(order, dims, dtype, iters);
}

extern "C" tvc_status hopm_backward(const void* A, int order, const int64_t* dims, void* const* x0, int iters,
                                    void* const* gx_final, const double* g_lambda, void* gA, void* const* gstart,
                                    tvc_dtype dtype, const float* slab_scales, void* workspace, size_t ws_bytes,
                                    tvc_stream_t stream) {
  if (!valid_dtype(dtype) || order < 2 || !A || !x0 || !gA || iters < 0) return TVC_ERR_INVALID_ARG;
  if (check_dims(order, dims, nullptr) != TVC_OK) return TVC_ERR_INVALID_ARG;
  const size_t vs = vec_size(dtype);
  if (!aligned(A, elem_size(dtype)) || !aligned(gA, vs)) return TVC_ERR_INVALID_ARG;
  for (int m = 0; m < order; m++)
    if (!x0[m] || !aligned(x0[m], vs)) return TVC_ERR_INVALID_ARG;
  return hopm_backward_launch(A, order, dims, x0, iters, gx_final, g_lambda, gA, gstart, dtype, slab_scales,
                              workspace, ws_bytes, (cudaStream_t)stream);
}
