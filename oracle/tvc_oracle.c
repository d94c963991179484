/*
 * Oracle for the tensor-vector contraction (TVC) and the higher-order power
 * method (HOPM).  TEST INFRASTRUCTURE ONLY: nothing in the library's product
 * path may call, link or load this file.  It is plain, slow and written to be
 * checked against the paper by eye: FP64 loop nests, no blocking, no fusion,
 * no reordering beyond what each definition states.  It shares no code with
 * the CUDA path.
 *
 * Paper: Martinez-Ferrer, Yzelman, Beltran, "Distributed and heterogeneous
 * tensor-vector contraction algorithms for high performance computing"
 * (arXiv 2501.03121).
 *
 * Storage (Section 3): dense tensors in last-order ("C row-major") layout,
 * zero-based indices, N = prod(n_i) elements.  The mode-k contraction
 * Y = A x_k x keeps the other d-1 modes; viewed through u = prod_{i<k} n_i
 * and v = prod_{i>k} n_i the tensor is a u x n_k x v array and
 *     Y[i][l] = sum_{j<n_k} A[i][j][l] x[j].
 *
 * Element types of A: FP64, FP32, BF16 (upper half of binary32), FP8 E4M3
 * (OCP 8-bit floating point, bias 7, max 448, no infinities) and FP16 (IEEE
 * 754 binary16, the "half" of Section 5.5's half-single format).  The
 * narrow types carry one FP32 scale per slab A[i_0, ...] (a NULL scale array
 * means 1); an element's value is scale[i_0] * decode(code), promoted to FP64
 * before any arithmetic (the storage-only use of low precision of Section
 * 5.5).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (IEEE semantics,
 * no fused multiply-add, no reassociation).
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_F64 0
#define OR_F32 1
#define OR_BF16 2
#define OR_E4M3 3
#define OR_F16 4

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_ZERO_NORM 5
#define OR_ERR_NONFINITE 6

#define OR_MAXD 16

/* Threads of the OpenMP loops that follow in the calling thread (the
 * outer-index "parallel for" of each routine); the results do not depend on
 * it.  Returns the previous count. */
int oracle_set_threads(int n) {
  int prev = omp_get_max_threads();
  if (n > 0) omp_set_num_threads(n);
  return prev;
}

/* ---------------------------------------------------------------- decoding */

/* BF16: the code is the upper 16 bits of a binary32 (Section 5.5). */
double oracle_decode_bf16(uint16_t code) {
  uint32_t bits = ((uint32_t)code) << 16;
  float f;
  memcpy(&f, &bits, 4);
  return (double)f;
}

/* E4M3 per the OCP FP8 definition: s.eeee.mmm, bias 7; e = 0 is subnormal
 * (m/8 * 2^-6); s.1111.111 is NaN; everything else (1 + m/8) * 2^(e-7). */
double oracle_decode_e4m3(uint8_t code) {
  int s = (code >> 7) & 1;
  int e = (code >> 3) & 15;
  int m = code & 7;
  double mag;
  if (e == 15 && m == 7) return NAN;
  if (e == 0)
    mag = ldexp((double)m / 8.0, -6);
  else
    mag = ldexp(1.0 + (double)m / 8.0, e - 7);
  return s ? -mag : mag;
}

/* IEEE 754 binary16: s.eeeee.mmmmmmmmmm, bias 15; e = 0 is subnormal
 * (m/1024 * 2^-14); e = 31 is infinity (m = 0) or NaN; everything else
 * (1 + m/1024) * 2^(e-15). */
double oracle_decode_f16(uint16_t code) {
  int s = (code >> 15) & 1;
  int e = (code >> 10) & 31;
  int m = code & 1023;
  double mag;
  if (e == 31) {
    if (m != 0) return NAN;
    mag = INFINITY;
  } else if (e == 0) {
    mag = ldexp((double)m / 1024.0, -14);
  } else {
    mag = ldexp(1.0 + (double)m / 1024.0, e - 15);
  }
  return s ? -mag : mag;
}

/* Value of element f of A, promoted to FP64.  slab = N / n_0. */
static double elem(int dtype, const void* A, const float* scales, int64_t slab, int64_t f) {
  switch (dtype) {
    case OR_F64: return ((const double*)A)[f];
    case OR_F32: return (double)((const float*)A)[f];
    case OR_BF16: return (double)scales[f / slab] * oracle_decode_bf16(((const uint16_t*)A)[f]);
    case OR_E4M3: return (double)scales[f / slab] * oracle_decode_e4m3(((const uint8_t*)A)[f]);
    case OR_F16: return (scales ? (double)scales[f / slab] : 1.0) * oracle_decode_f16(((const uint16_t*)A)[f]);
  }
  return NAN;
}

static int valid_shape(int order, const int64_t* dims) {
  if (order < 1 || order > OR_MAXD) return 0;
  for (int i = 0; i < order; i++)
    if (dims[i] < 1) return 0;
  return 1;
}

static int64_t prod(const int64_t* dims, int lo, int hi) {
  int64_t p = 1;
  for (int i = lo; i < hi; i++) p *= dims[i];
  return p;
}

/* -------------------------------------------------------------------- TVC */

/* Y := alpha * (A x_k x) + beta * Y (Section 3 definition, with the BLAS-like
 * scalars of Eq. 1 for p = 1).  beta == 0 means Y is not read.  x has n_k
 * entries, Y has u*v entries in row-major order of the remaining modes. */
int oracle_tvc(int dtype, const void* A, const float* scales, int order, const int64_t* dims,
               int mode, const double* x, double* y, double alpha, double beta) {
  if (!valid_shape(order, dims) || mode < 0 || mode >= order) return OR_ERR_ARG;
  int64_t u = prod(dims, 0, mode), nk = dims[mode], v = prod(dims, mode + 1, order);
  int64_t slab = prod(dims, 1, order);
  int64_t nout = u * v;
#pragma omp parallel for schedule(static)
  for (int64_t o = 0; o < nout; o++) {
    int64_t i = o / v, l = o % v;
    double s = 0.0;
    for (int64_t j = 0; j < nk; j++) s += elem(dtype, A, scales, slab, (i * nk + j) * v + l) * x[j];
    y[o] = (beta != 0.0) ? alpha * s + beta * y[o] : alpha * s;
  }
  return OR_OK;
}

/* The same contraction with error-free transformations, for measuring the
 * error of another arithmetic against the exact sum: every product a*x is
 * split exactly into p + e by one fused multiply-add (TwoProduct:
 * e = fma(a, x, -p)), the p are added with Knuth's TwoSum (each rounding
 * error recovered exactly) and every recovered error and every e is summed
 * in a second accumulator; the result is the two accumulators added once.
 * This is the compensated dot product "Dot2" of Ogita, Rump and Oishi
 * (Accurate sum and dot product, SIAM J. Sci. Comput. 26, 2005): its error is
 * at most 2^-53 |y| + (n 2^-53)^2 / (1 - n 2^-53)^2 * sum_j |a_j x_j|, i.e.
 * the exact sum rounded once unless n is astronomically large.  alpha = 1,
 * beta = 0.  fma() is the C99 correctly rounded fused multiply-add (the
 * explicit call is not affected by -ffp-contract=off). */
int oracle_tvc_exact(int dtype, const void* A, const float* scales, int order, const int64_t* dims,
                     int mode, const double* x, double* y) {
  if (!valid_shape(order, dims) || mode < 0 || mode >= order) return OR_ERR_ARG;
  int64_t u = prod(dims, 0, mode), nk = dims[mode], v = prod(dims, mode + 1, order);
  int64_t slab = prod(dims, 1, order);
  int64_t nout = u * v;
#pragma omp parallel for schedule(static)
  for (int64_t o = 0; o < nout; o++) {
    int64_t i = o / v, l = o % v;
    double s = 0.0, c = 0.0;
    for (int64_t j = 0; j < nk; j++) {
      double a = elem(dtype, A, scales, slab, (i * nk + j) * v + l);
      double p = a * x[j];
      double e = fma(a, x[j], -p);
      double t = s + p;
      double bp = t - s;
      double err = (s - (t - bp)) + (p - bp);
      s = t;
      c = c + (err + e);
    }
    y[o] = s + c;
  }
  return OR_OK;
}

/* -------------------------------------------------------------------- TMC */

/* Tensor-matrix contraction in mode k (the TMC of Section 1, the mode-k
 * product with a matrix): X is an R x n_k matrix in row-major order and
 *     Y[i][r][l] = alpha * sum_{j<n_k} A[i][j][l] X[r][j] + beta * Y[i][r][l],
 * i.e. Y has the shape of A with n_k replaced by R, row-major.  Row r of X
 * gives the mode-k TVC with that row.  beta == 0 means Y is not read. */
int oracle_tmc(int dtype, const void* A, const float* scales, int order, const int64_t* dims, int mode,
               const double* X, int64_t R, double* Y, double alpha, double beta) {
  if (!valid_shape(order, dims) || mode < 0 || mode >= order || R < 1) return OR_ERR_ARG;
  int64_t u = prod(dims, 0, mode), nk = dims[mode], v = prod(dims, mode + 1, order);
  int64_t slab = prod(dims, 1, order);
  int64_t nout = u * R * v;
#pragma omp parallel for schedule(static)
  for (int64_t o = 0; o < nout; o++) {
    int64_t i = o / (R * v), r = (o / v) % R, l = o % v;
    double s = 0.0;
    for (int64_t j = 0; j < nk; j++) s += elem(dtype, A, scales, slab, (i * nk + j) * v + l) * X[r * nk + j];
    Y[o] = (beta != 0.0) ? alpha * s + beta * Y[o] : alpha * s;
  }
  return OR_OK;
}

/* ------------------------------------------------- Khatri-Rao and MTTKRP */

/* Khatri-Rao product (Section 1) of `count` matrices U_m (rows[m] x R,
 * row-major): the columnwise Kronecker product, out[(i_0, ..., i_{c-1})][r] =
 * prod_m U_m[i_m][r] with i_0 the most significant index of the row
 * (rows = prod rows[m]; count == 0 gives one row of ones). */
int oracle_khatri_rao(const double* const* U, int count, const int64_t* rows, int64_t R, double* out) {
  if (count < 0 || R < 1) return OR_ERR_ARG;
  int64_t n = 1;
  for (int m = 0; m < count; m++) {
    if (rows[m] < 1) return OR_ERR_ARG;
    n *= rows[m];
  }
  for (int64_t row = 0; row < n; row++) {
    for (int64_t r = 0; r < R; r++) out[row * R + r] = 1.0;
    int64_t rem = row;
    for (int m = count - 1; m >= 0; m--) {
      int64_t im = rem % rows[m];
      rem /= rows[m];
      for (int64_t r = 0; r < R; r++) out[row * R + r] *= U[m][im * R + r];
    }
  }
  return OR_OK;
}

/* Matricized tensor times Khatri-Rao product for mode k (the core of CP
 * alternating least squares, Section 1): with factor matrices X_m (n_m x R,
 * row-major) for every m != k,
 *     M[i_k][r] = sum over all other indices of A[i_0..i_{d-1}] prod_{m != k} X_m[i_m][r].
 * factors[k] is not read.  M is n_k x R, row-major.  Straight from the
 * definition: one pass over the elements, each weighted by its row of the
 * Khatri-Rao product of the other factors. */
int oracle_mttkrp(int dtype, const void* A, const float* scales, int order, const int64_t* dims, int mode,
                  const double* const* factors, int64_t R, double* M) {
  if (!valid_shape(order, dims) || mode < 0 || mode >= order || R < 1) return OR_ERR_ARG;
  for (int m = 0; m < order; m++)
    if (m != mode && !factors[m]) return OR_ERR_ARG;
  int64_t N = prod(dims, 0, order), slab = prod(dims, 1, order);
  for (int64_t q = 0; q < dims[mode] * R; q++) M[q] = 0.0;
  double* w = (double*)malloc(sizeof(double) * (size_t)R);
  if (!w) return OR_ERR_ARG;
  for (int64_t f = 0; f < N; f++) {
    double a = elem(dtype, A, scales, slab, f);
    int64_t rem = f, ik = 0;
    for (int64_t r = 0; r < R; r++) w[r] = 1.0;
    for (int m = order - 1; m >= 0; m--) {
      int64_t im = rem % dims[m];
      rem /= dims[m];
      if (m == mode) {
        ik = im;
        continue;
      }
      for (int64_t r = 0; r < R; r++) w[r] *= factors[m][im * R + r];
    }
    for (int64_t r = 0; r < R; r++) M[ik * R + r] += a * w[r];
  }
  free(w);
  return OR_OK;
}

/* ---------------------------------------------------------- TVC gradients */

/* Gradient of L(Y) with Y = A x_k x, with respect to x:
 *     gx[j] = sum_{i,l} A[i][j][l] * gy[i][l]. */
int oracle_tvc_grad_x(int dtype, const void* A, const float* scales, int order, const int64_t* dims,
                      int mode, const double* gy, double* gx) {
  if (!valid_shape(order, dims) || mode < 0 || mode >= order) return OR_ERR_ARG;
  int64_t u = prod(dims, 0, mode), nk = dims[mode], v = prod(dims, mode + 1, order);
  int64_t slab = prod(dims, 1, order);
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < nk; j++) {
    double s = 0.0;
    for (int64_t i = 0; i < u; i++)
      for (int64_t l = 0; l < v; l++) s += elem(dtype, A, scales, slab, (i * nk + j) * v + l) * gy[i * v + l];
    gx[j] = s;
  }
  return OR_OK;
}

/* Gradient with respect to A: gA[i][j][l] = gy[i][l] * x[j] (rank-1). */
int oracle_tvc_grad_A(int order, const int64_t* dims, int mode, const double* x, const double* gy,
                      double* gA) {
  if (!valid_shape(order, dims) || mode < 0 || mode >= order) return OR_ERR_ARG;
  int64_t u = prod(dims, 0, mode), nk = dims[mode], v = prod(dims, mode + 1, order);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < u; i++)
    for (int64_t j = 0; j < nk; j++)
      for (int64_t l = 0; l < v; l++) gA[(i * nk + j) * v + l] = gy[i * v + l] * x[j];
  return OR_OK;
}

/* ------------------------------------------------------------------ HOPM */

/* A working tensor of the power method: its data (FP64, or the typed input
 * tensor when `typed` is set), the original mode ids it still carries, and
 * their sizes.  Contracted modes are dropped (they would be of size one). */
typedef struct {
  int typed;
  int dtype;
  const void* A;
  const float* scales;
  int64_t slab;
  double* data;
  int nd;
  int modes[OR_MAXD];
  int64_t dims[OR_MAXD];
} otensor;

static int64_t osize(const otensor* t) { return prod(t->dims, 0, t->nd); }

/* out = t x_m x_m (m is an ORIGINAL mode id that t still carries).
 * Counts touched elements: the whole input, the whole output, the vector. */
static int ocontract(const otensor* t, int m, const double* xm, otensor* out, int64_t* touched) {
  int p = -1;
  for (int q = 0; q < t->nd; q++)
    if (t->modes[q] == m) p = q;
  if (p < 0) return OR_ERR_ARG;
  int64_t u = prod(t->dims, 0, p), nk = t->dims[p], v = prod(t->dims, p + 1, t->nd);
  out->typed = 0;
  out->nd = t->nd - 1;
  for (int q = 0, r = 0; q < t->nd; q++)
    if (q != p) {
      out->modes[r] = t->modes[q];
      out->dims[r] = t->dims[q];
      r++;
    }
  out->data = (double*)malloc(sizeof(double) * (size_t)(u * v));
  if (!out->data) return OR_ERR_ARG;
  if (t->typed) {
    oracle_tvc(t->dtype, t->A, t->scales, t->nd, t->dims, p, xm, out->data, 1.0, 0.0);
  } else {
    oracle_tvc(OR_F64, t->data, NULL, t->nd, t->dims, p, xm, out->data, 1.0, 0.0);
  }
  if (touched) *touched += osize(t) + u * v + nk;
  return OR_OK;
}

static void ofree(otensor* t) {
  if (!t->typed && t->data) free(t->data);
  t->data = NULL;
}

/* Normalisation x_j <- T / ||T||_2 (FP64).  Reads T twice and writes x_j:
 * the 3 n term of Eq. 3.  Returns the norm through *sigma. */
static int onormalise(const double* T, int64_t n, double* xj, double* sigma, int64_t* touched) {
  double ss = 0.0;
  for (int64_t i = 0; i < n; i++) ss += T[i] * T[i];
  double s = sqrt(ss);
  if (touched) *touched += 3 * n;
  *sigma = s;
  if (!isfinite(s)) return OR_ERR_NONFINITE;
  if (s == 0.0) return OR_ERR_ZERO_NORM;
  for (int64_t i = 0; i < n; i++) xj[i] = T[i] / s;
  return OR_OK;
}

static void base_tensor(otensor* t, int dtype, const void* A, const float* scales, int order,
                        const int64_t* dims) {
  t->typed = 1;
  t->dtype = dtype;
  t->A = A;
  t->scales = scales;
  t->slab = prod(dims, 1, order);
  t->data = NULL;
  t->nd = order;
  for (int q = 0; q < order; q++) {
    t->modes[q] = q;
    t->dims[q] = dims[q];
  }
}

/* Stopping rule (the paper states none): after sweep t >= 2 stop when
 * tol > 0 and |lambda_t - lambda_{t-1}| <= tol * lambda_t. */
static int converged(double lam, double prev, int t, double tol) {
  if (t < 2 || !(tol > 0.0)) return 0;
  double scale = lam > 1e-300 ? lam : 1e-300;
  return fabs(lam - prev) <= tol * scale;
}

/* Canonical (two-buffer) Gauss-Seidel HOPM, Section 3: in each sweep, for
 * every external mode j = 0..d-1 in ascending order, contract A with every
 * other x_m in ascending m, normalise the resulting n_j-vector into x_j.
 * lambda_t = the norm of the last update (j = d-1) of sweep t.
 * x holds x_0..x_{d-1} back to back (in/out).  x_0's input value is unused.
 * touched (nullable) accumulates Eq. 3's streamed-element count per sweep:
 * entry t-1 gets sweep t's count.  tvcs (nullable) counts contractions. */
int oracle_hopm(int dtype, const void* A, const float* scales, int order, const int64_t* dims,
                double* x, int iters, double tol, double* lambda_out, int* sweeps_out,
                double* lambda_hist, int64_t* touched, int64_t* tvcs) {
  if (!valid_shape(order, dims) || order < 2 || iters < 0) return OR_ERR_ARG;
  int64_t off[OR_MAXD + 1];
  off[0] = 0;
  for (int m = 0; m < order; m++) off[m + 1] = off[m] + dims[m];
  double lam = 0.0, prev = 0.0;
  int status = OR_OK, t;
  for (t = 1; t <= iters; t++) {
    int64_t tc = 0;
    for (int j = 0; j < order && status == OR_OK; j++) {
      otensor cur;
      base_tensor(&cur, dtype, A, scales, order, dims);
      for (int m = 0; m < order; m++) {
        if (m == j) continue;
        otensor nxt;
        status = ocontract(&cur, m, x + off[m], &nxt, &tc);
        ofree(&cur);
        cur = nxt;
        if (tvcs) (*tvcs)++;
        if (status != OR_OK) break;
      }
      if (status != OR_OK) {
        ofree(&cur);
        break;
      }
      double sigma;
      status = onormalise(cur.data, dims[j], x + off[j], &sigma, &tc);
      ofree(&cur);
      if (j == order - 1 && status == OR_OK) lam = sigma;
    }
    if (touched) touched[t - 1] = tc;
    if (status != OR_OK) break;
    if (lambda_hist) lambda_hist[t - 1] = lam;
    if (converged(lam, prev, t, tol)) {
      prev = lam;
      break;
    }
    prev = lam;
  }
  if (lambda_out) *lambda_out = lam;
  if (sweeps_out) *sweeps_out = (t > iters) ? iters : t;
  return status;
}

/* Jacobi HOPM (a variant of the power method, not the paper's Algorithm 1):
 * in each sweep every z_j = A x_{m != j} x_m is formed from the vectors of
 * the PREVIOUS sweep (canonical chain, every other mode ascending), then
 * every x_j <- z_j / ||z_j||.  lambda_t = ||z_{d-1}|| of sweep t (as for the
 * Gauss-Seidel method); same stopping rule, outputs and status.  All d
 * updates read the same vectors, so one pass over A can serve a sweep. */
int oracle_hopm_jacobi(int dtype, const void* A, const float* scales, int order, const int64_t* dims,
                       double* x, int iters, double tol, double* lambda_out, int* sweeps_out,
                       double* lambda_hist) {
  if (!valid_shape(order, dims) || order < 2 || iters < 0) return OR_ERR_ARG;
  int64_t off[OR_MAXD + 1];
  off[0] = 0;
  for (int m = 0; m < order; m++) off[m + 1] = off[m] + dims[m];
  double* z = (double*)malloc(sizeof(double) * (size_t)off[order]);
  if (!z) return OR_ERR_ARG;
  double lam = 0.0, prev = 0.0;
  int status = OR_OK, t;
  for (t = 1; t <= iters; t++) {
    for (int j = 0; j < order && status == OR_OK; j++) {
      otensor cur;
      base_tensor(&cur, dtype, A, scales, order, dims);
      for (int m = 0; m < order; m++) {
        if (m == j) continue;
        otensor nxt;
        status = ocontract(&cur, m, x + off[m], &nxt, NULL);
        ofree(&cur);
        cur = nxt;
        if (status != OR_OK) break;
      }
      if (status == OR_OK) memcpy(z + off[j], cur.data, sizeof(double) * (size_t)dims[j]);
      ofree(&cur);
    }
    for (int j = 0; j < order && status == OR_OK; j++) {
      double sigma;
      status = onormalise(z + off[j], dims[j], x + off[j], &sigma, NULL);
      if (j == order - 1 && status == OR_OK) lam = sigma;
    }
    if (status != OR_OK) break;
    if (lambda_hist) lambda_hist[t - 1] = lam;
    if (converged(lam, prev, t, tol)) {
      prev = lam;
      break;
    }
    prev = lam;
  }
  free(z);
  if (lambda_out) *lambda_out = lam;
  if (sweeps_out) *sweeps_out = (t > iters) ? iters : t;
  return status;
}

/* Three-buffer HOPM of Algorithm 1 for one process (p = 1): the external
 * iteration j reuses the prefix W_{j-1} = A x_0 x_0 ... x_{j-2} x_{j-2}
 * (ORIGINAL mode ids throughout).  Per iteration j, with
 *     a = (j > 0 ? 0 : 1),  mu = max(a, j),  nu = (j < d-1 ? d-1 : d-2):
 *   j < 2 :  Y_a := W_j <- A x_a x_a
 *   j >= 2:  Y_{mu-1} := W_j <- W_{j-1} x_{mu-1} x_{mu-1}
 *   Y_{mu+1} <- Y_{mu+a-1} x_{mu+1} x_{mu+1}     (skipped when mu+1 > d-1)
 *   Y_k <- Y_{k-1} x_k x_k for k = mu+2 .. nu
 *   x_j <- Y_nu / ||Y_nu||.
 * The skip of the second step when mu+1 > d-1 is the reading under which the
 * algorithm saves (d-1)(d-2)/2 contractions per sweep.  Same stopping rule,
 * outputs and counters as oracle_hopm. */
int oracle_hopm3(int dtype, const void* A, const float* scales, int order, const int64_t* dims,
                 double* x, int iters, double tol, double* lambda_out, int* sweeps_out,
                 double* lambda_hist, int64_t* touched, int64_t* tvcs) {
  if (!valid_shape(order, dims) || order < 2 || iters < 0) return OR_ERR_ARG;
  int d = order;
  int64_t off[OR_MAXD + 1];
  off[0] = 0;
  for (int m = 0; m < d; m++) off[m + 1] = off[m] + dims[m];
  double lam = 0.0, prev = 0.0;
  int status = OR_OK, t;
  otensor Abase;
  base_tensor(&Abase, dtype, A, scales, order, dims);
  for (t = 1; t <= iters; t++) {
    int64_t tc = 0;
    otensor W;  /* W_{j-1}, carried from iteration j-1 */
    W.typed = 0;
    W.data = NULL;
    for (int j = 0; j < d && status == OR_OK; j++) {
      int a = (j > 0) ? 0 : 1;
      int mu = (a > j) ? a : j;
      int nu = (j < d - 1) ? d - 1 : d - 2;
      otensor Y[OR_MAXD + 1];
      int have[OR_MAXD + 1];
      memset(have, 0, sizeof(have));
      otensor Wj;
      if (j < 2) {
        status = ocontract(&Abase, a, x + off[a], &Wj, &tc);
      } else {
        status = ocontract(&W, mu - 1, x + off[mu - 1], &Wj, &tc);
      }
      if (tvcs) (*tvcs)++;
      if (status != OR_OK) break;
      int widx = (j < 2) ? a : mu - 1;
      Y[widx] = Wj; /* aliases W_j: not freed through Y */
      have[widx] = 2;
      if (mu + 1 <= d - 1) {
        int src = mu + a - 1;
        status = ocontract(&Y[src], mu + 1, x + off[mu + 1], &Y[mu + 1], &tc);
        if (tvcs) (*tvcs)++;
        if (status == OR_OK) have[mu + 1] = 1;
      }
      for (int k = mu + 2; k <= nu && status == OR_OK; k++) {
        status = ocontract(&Y[k - 1], k, x + off[k], &Y[k], &tc);
        if (tvcs) (*tvcs)++;
        if (status == OR_OK) have[k] = 1;
      }
      double sigma = 0.0;
      if (status == OR_OK) status = onormalise(Y[nu].data, dims[j], x + off[j], &sigma, &tc);
      if (j == d - 1 && status == OR_OK) lam = sigma;
      for (int k = 0; k <= d; k++)
        if (have[k] == 1) ofree(&Y[k]);
      ofree(&W);
      W = Wj;
    }
    ofree(&W);
    if (touched) touched[t - 1] = tc;
    if (status != OR_OK) break;
    if (lambda_hist) lambda_hist[t - 1] = lam;
    if (converged(lam, prev, t, tol)) {
      prev = lam;
      break;
    }
    prev = lam;
  }
  if (lambda_out) *lambda_out = lam;
  if (sweeps_out) *sweeps_out = (t > iters) ? iters : t;
  return status;
}

/* --------------------------------------------------------------- storage */

/* Round-to-nearest-even of a binary32 to BF16 (upper 16 bits).  With
 * truncate != 0 the lower half is simply dropped, the paper's "brain"
 * conversion (Section 5.5).  NaN maps to 0x7FC0 with the input's sign. */
uint16_t oracle_bf16_from_f32(float f, int truncate) {
  uint32_t b;
  memcpy(&b, &f, 4);
  if (isnan(f)) return (uint16_t)(((b >> 16) & 0x8000u) | 0x7FC0u);
  if (truncate) return (uint16_t)(b >> 16);
  uint32_t lsb = (b >> 16) & 1u;
  b += 0x7FFFu + lsb;
  return (uint16_t)(b >> 16);
}

/* Round a binary32 to E4M3 to nearest, ties to even, saturating to +-448
 * (OCP "satfinite" conversion); NaN -> 0x7F.  The E4M3 magnitudes in code
 * order form a grid whose spacing is 2^-9 below 2^-6 and 2^(e-3) in the
 * binade [2^e, 2^(e+1)); the code of a magnitude is its grid index. */
uint8_t oracle_e4m3_from_f32(float f) {
  if (isnan(f)) return 0x7F;
  uint8_t s = signbit(f) ? 0x80 : 0x00;
  double a = fabs((double)f);
  if (a >= 448.0) return s | 0x7E;
  double r;
  int code;
  if (a < ldexp(1.0, -6)) {
    r = nearbyint(a / ldexp(1.0, -9)); /* 0..8, exact quotient */
    code = (int)r;
  } else {
    int e2;
    frexp(a, &e2); /* a = f * 2^e2, f in [0.5, 1): binade exponent e = e2-1 */
    int e = e2 - 1;
    r = nearbyint(a / ldexp(1.0, e - 3)); /* 8..16 */
    if (r >= 16.0) {
      e += 1;
      r = 8.0;
    }
    code = ((e + 7) << 3) | ((int)r - 8);
    if (code > 0x7E) code = 0x7E;
  }
  return (uint8_t)(s | code);
}

/* -------------------------------------------- distributed byte model */

/* Touched elements of ONE process in external iteration j of the
 * distributed HOPM (Section 4.2) on a hypersquare tensor n^d split along
 * dimension s over p processes with n divisible by p, counted as in Eq. 3:
 * a contraction touches its whole input, its whole output and the part of
 * the vector it uses; the normalisation touches 3 x the length the process
 * normalises (n/p for j = s, whose pieces are gathered afterwards; n for
 * j != s, after the sum over processes).  Inter-process traffic is not
 * counted (as in Eq. 4-7).  Sizes only: no arithmetic.
 *   three = 0: the canonical chain (every other mode, ascending, from A);
 *   three = 1: Algorithm 1's chain (the prefix W carried from iteration
 *              j-1; iterations 0..j-1 are walked to rebuild it, only
 *              iteration j is counted).
 * Returns -1 for invalid arguments. */
static int64_t dm_size(const int64_t* sz, int d) { return prod(sz, 0, d); }

static void dm_contract(const int64_t* in, int d, int m, int64_t* out, int64_t* touched) {
  int64_t isz = dm_size(in, d);
  for (int q = 0; q < d; q++) out[q] = in[q];
  out[m] = 1; /* the contracted mode keeps size one */
  if (touched) *touched += isz + isz / in[m] + in[m];
}

int64_t oracle_dhopm_touched(int d, int64_t n, int p, int s, int j, int three) {
  if (d < 2 || d > OR_MAXD || n < 1 || p < 1 || n % p != 0 || s < 0 || s >= d || j < 0 || j >= d) return -1;
  int64_t base[OR_MAXD];
  for (int q = 0; q < d; q++) base[q] = n;
  base[s] = n / p;
  int64_t t = 0;
  const int64_t vec_len = (j == s) ? n / p : n;
  if (!three) {
    int64_t cur[OR_MAXD], nxt[OR_MAXD];
    memcpy(cur, base, sizeof(int64_t) * (size_t)d);
    for (int m = 0; m < d; m++) {
      if (m == j) continue;
      dm_contract(cur, d, m, nxt, &t);
      memcpy(cur, nxt, sizeof(int64_t) * (size_t)d);
    }
    return t + 3 * vec_len;
  }
  int64_t W[OR_MAXD];
  for (int jj = 0; jj <= j; jj++) {
    int64_t* tc = (jj == j) ? &t : NULL;
    int a = (jj > 0) ? 0 : 1;
    int mu = (a > jj) ? a : jj;
    int nu = (jj < d - 1) ? d - 1 : d - 2;
    int64_t Y[OR_MAXD + 1][OR_MAXD];
    int64_t Wj[OR_MAXD];
    if (jj < 2)
      dm_contract(base, d, a, Wj, tc);
    else
      dm_contract(W, d, mu - 1, Wj, tc);
    int widx = (jj < 2) ? a : mu - 1;
    memcpy(Y[widx], Wj, sizeof(int64_t) * (size_t)d);
    if (mu + 1 <= d - 1) dm_contract(Y[mu + a - 1], d, mu + 1, Y[mu + 1], tc);
    for (int k = mu + 2; k <= nu; k++) dm_contract(Y[k - 1], d, k, Y[k], tc);
    memcpy(W, Wj, sizeof(int64_t) * (size_t)d);
  }
  return t + 3 * vec_len;
}

/* binary32 -> binary16, round to nearest, ties to even (IEEE 754), by
 * value: |f| >= 65520 (halfway between the largest finite half, 65504, and
 * 2^16) becomes infinity; below 2^-14 the quantum is 2^-24 (subnormals);
 * NaN stays NaN (quiet, sign kept). */
uint16_t oracle_f16_from_f32(float f) {
  uint16_t s = signbit(f) ? 0x8000 : 0;
  double a = fabs((double)f);
  if (isnan(f)) return (uint16_t)(s | 0x7E00);
  if (a >= 65520.0) return (uint16_t)(s | 0x7C00);
  if (a < ldexp(1.0, -14)) {
    double q = nearbyint(a / ldexp(1.0, -24)); /* 0..1024; 1024 is the smallest normal */
    return (uint16_t)(s | (uint16_t)q);
  }
  int ex;
  frexp(a, &ex); /* a = fr * 2^ex, fr in [0.5, 1) */
  int e = ex - 1;
  double r = nearbyint(a / ldexp(1.0, e - 10)); /* 1024..2048 */
  if (r >= 2048.0) {
    e += 1;
    r = 1024.0;
  }
  return (uint16_t)(s | ((e + 15) << 10) | ((int)r - 1024));
}

/* Per-slab quantisation of an FP32 tensor (slab = A[i_0, ...], N/n_0
 * elements).  E4M3: scale = amax(slab) / 448 in FP32 (1 when the slab is all
 * zero), code = E4M3(value / scale) with the FP32 quotient.  BF16: scale = 1,
 * code = BF16(value) (RNE, or truncation when truncate != 0).  F16: scale =
 * 1, code = binary16(value) (RNE); every code is written and the status is
 * OR_ERR_NONFINITE when some code is infinite or NaN (overflow or a
 * non-finite source). */
int oracle_quantise(int dtype, const float* src, int order, const int64_t* dims, void* codes,
                    float* scales, int truncate) {
  if (!valid_shape(order, dims)) return OR_ERR_ARG;
  if (dtype != OR_BF16 && dtype != OR_E4M3 && dtype != OR_F16) return OR_ERR_ARG;
  if (dtype == OR_F16) {
    int64_t n0 = dims[0], slab = prod(dims, 1, order);
    int bad = 0;
    for (int64_t i = 0; i < n0; i++) scales[i] = 1.0f;
    for (int64_t f = 0; f < n0 * slab; f++) {
      uint16_t c = oracle_f16_from_f32(src[f]);
      ((uint16_t*)codes)[f] = c;
      if ((c & 0x7C00) == 0x7C00) bad = 1;
    }
    return bad ? OR_ERR_NONFINITE : OR_OK;
  }
  int64_t n0 = dims[0], slab = prod(dims, 1, order);
  for (int64_t i = 0; i < n0; i++) {
    const float* p = src + i * slab;
    float sc = 1.0f;
    if (dtype == OR_E4M3) {
      float amax = 0.0f;
      for (int64_t f = 0; f < slab; f++) {
        float a = fabsf(p[f]);
        if (!(a <= amax)) amax = a; /* NaN propagates */
      }
      if (!isfinite(amax)) return OR_ERR_NONFINITE;
      if (amax > 0.0f) sc = amax / 448.0f;
    }
    scales[i] = sc;
    for (int64_t f = 0; f < slab; f++) {
      if (dtype == OR_E4M3)
        ((uint8_t*)codes)[i * slab + f] = oracle_e4m3_from_f32(p[f] / sc);
      else
        ((uint16_t*)codes)[i * slab + f] = oracle_bf16_from_f32(p[f], truncate);
    }
  }
  return OR_OK;
}
