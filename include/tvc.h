/*
 * tvc.h -- C ABI of the GB300 tensor-vector contraction library.
 *
 * Method: Martinez-Ferrer, Yzelman, Beltran, "Distributed and heterogeneous
 * tensor-vector contraction algorithms for high performance computing"
 * (arXiv 2501.03121).  This library is the single-GPU hot path of that
 * method: the mode-oblivious dense tensor-vector contraction (TVC) and the
 * higher-order power method (HOPM) built on it, with low-precision storage,
 * adjoints and batching; the 1D split over virtual ranks (Eq. 1/2,
 * Algorithm 1); and the building blocks that Section 1 names next to the
 * TVC: the tensor-matrix contraction, the Khatri-Rao product and the MTTKRP
 * of CP alternating least squares.
 *
 * Entry points: tvc, tvc_ex, tvc_noalloc; tvc_quantise; tvc_backward;
 * hopm, hopm_jacobi, hopm_backward; tvc_batched, tvc_batched_autotune,
 * hopm_batched; tvc_split_1d, tvc_slab_copy, dtvc, dhopm; tmc, khatri_rao,
 * mttkrp; each with its *_workspace_size query where it takes a workspace;
 * diagnostics tvc_read_status, tvc_status_string, tvc_kernel_launches,
 * tvc_device_error.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Layout (Section 3): a d-order tensor A of sizes n_0 x ... x n_{d-1} is
 *   stored dense in last-order ("C row-major") layout, zero-based, with
 *   N = prod n_i elements.  For mode k, u = prod_{i<k} n_i and
 *   v = prod_{i>k} n_i, and A is read as a u x n_k x v array.
 * Pointers: A, x, y and every vector/workspace argument are DEVICE pointers
 *   (memory the caller owns, e.g. from torch); dims and the descriptor arrays
 *   of the batched calls are HOST pointers read before the call returns.
 *   Tensors must be element-aligned; 16-byte alignment enables wider loads.
 * Types: tvc_dtype names the storage of A.  Vectors (x, y, gradients,
 *   prefix tensors) are FP64 for TVC_F64 and TVC_F32D and FP32 for every
 *   other type.  TVC_F32D (Section 5.5's single-double) reads binary32
 *   elements and computes in FP64 like TVC_F64.
 *   TVC_BF16, TVC_E4M3 and TVC_F16 carry one FP32 scale per slab A[i_0, ...]
 *   (n_0 scales, device memory); an element's value is
 *   scale[i_0] * decode(code).  A NULL scale pointer means all scales are 1.
 * Streams: every call is stream-ordered on `stream` (NULL = legacy default
 *   stream) and returns without synchronising.  Argument errors are
 *   detected on the host before anything is launched and are returned
 *   synchronously; numerical conditions found on the device (zero norm,
 *   non-finite values) are written to a device status word where the call
 *   has one.
 * Sizes: 1 <= order <= TVC_MAX_ORDER, every n_i >= 1, N < 2^62; all
 *   indexing is 64-bit.
 * Aliasing: outputs must not overlap inputs.
 * Threading: calls on different streams may run concurrently when they use
 *   different workspaces (tvc() takes its own per call; tvc_noalloc shares
 *   one array per device and must be ordered).
 */
#ifndef TVC_GB300_H
#define TVC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TVC_MAX_ORDER 16

/* Same object as cudaStream_t, declared without the CUDA headers. */
typedef struct CUstream_st* tvc_stream_t;

typedef enum {
  TVC_F64 = 0,  /* binary64 storage, FP64 results                        */
  TVC_F32 = 1,  /* binary32 storage, FP32 accumulation                   */
  TVC_BF16 = 2, /* upper half of binary32, per-slab FP32 scale           */
  TVC_E4M3 = 3, /* OCP FP8 E4M3 (bias 7, max 448), per-slab FP32 scale   */
  TVC_F16 = 4,  /* IEEE binary16 (Section 5.5's half-single), FP32 math  */
  TVC_F32D = 5  /* binary32 storage, FP64 arithmetic (single-double)     */
} tvc_dtype;

typedef enum {
  TVC_OK = 0,
  TVC_ERR_INVALID_ARG = 1, /* bad pointer, order, size, mode or dtype         */
  TVC_ERR_UNSUPPORTED = 2, /* valid but not supported by this library         */
  TVC_ERR_WORKSPACE = 3,   /* workspace smaller than the *_workspace_size     */
  TVC_ERR_CUDA = 4,        /* a CUDA launch or runtime call failed            */
  TVC_ERR_ZERO_NORM = 5,   /* device status: a HOPM update had zero norm      */
  TVC_ERR_NONFINITE = 6,   /* device status: NaN or Inf met in a norm         */
  TVC_ERR_TIMEOUT = 7      /* device status: a bounded device wait gave up    */
} tvc_status;

/* Human-readable name of a status code (static string). */
const char* tvc_status_string(tvc_status s);

/* ------------------------------------------------------------------ TVC */

/*
 * Y = A x_mode x  (Section 3, "k-mode contraction"):
 *     y[i*v + l] = sum_{j < n_k} A[(i*n_k + j)*v + l] * x[j]
 * x: n_mode entries; y: N / n_mode entries, the remaining modes in
 * row-major order (the contracted mode behaves as a mode of size one).
 * Narrow types use unit scales.
 * Scratch: shapes that need a workspace (FP64 always: the split pieces of
 * x; any type when n_mode is split over several blocks) take it for the
 * duration of the call from a library-owned memory pool of the current
 * device, stream-ordered: cudaMallocFromPoolAsync on `stream` before the
 * kernels and cudaFreeAsync on `stream` after them.  So calls on different
 * streams never share scratch and may run concurrently; no call
 * synchronises the device or the stream.  The pool is created by the
 * first call on a device that needs scratch (make that call before any
 * stream capture); it keeps the memory it has handed out reserved for
 * later calls until the process exits.  Under stream capture the
 * allocation and the free become the graph's own memory nodes, so the call
 * can be captured in a CUDA graph.  tvc_ex with a caller-owned workspace
 * allocates nothing.
 */
tvc_status tvc(const void* A, int order, const int64_t* dims, int mode, const void* x, void* y,
               tvc_dtype dtype, tvc_stream_t stream);

/*
 * Y := alpha * (A x_mode x) + beta * Y  (the BLAS-like form of Eq. 1 for a
 * single process).  beta == 0 means y is not read (NaN in y is ignored).
 * slab_scales: n_0 FP32 scales for TVC_BF16 / TVC_E4M3 / TVC_F16, ignored otherwise.
 * workspace: device memory of at least tvc_workspace_size(...) bytes; it
 * may be NULL when that size is 0.  Returns TVC_ERR_WORKSPACE if too small.
 */
tvc_status tvc_ex(const void* A, int order, const int64_t* dims, int mode, const void* x, void* y,
                  tvc_dtype dtype, const float* slab_scales, double alpha, double beta,
                  void* workspace, size_t ws_bytes, tvc_stream_t stream);

/* Bytes of workspace tvc_ex needs for this shape (0 when none); the same
 * plan is used by tvc_ex for the same arguments on the same device. */
size_t tvc_workspace_size(int order, const int64_t* dims, int mode, tvc_dtype dtype);

/*
 * Mode-k tensor-matrix contraction (TMC, Section 1; the mode-k product with
 * a matrix that the higher-order orthogonal iteration for the Tucker
 * decomposition and CP alternating least squares are built from):
 *     Y[i][r][l] := alpha * sum_{j < n_mode} A[i][j][l] X[r][j] + beta * Y[i][r][l]
 * with A read as u x n_mode x v (Section 3).  X: R x n_mode matrix, row-major,
 * FP64 for TVC_F64 / TVC_F32D and FP32 otherwise.  Y: the dims of A with
 * n_mode replaced by R, row-major, same type as X; beta == 0 means Y is not
 * read.  Row r of Y (along mode) is the TVC of A with row r of X.  A is read
 * once per pass of up to 16 rows of X (8 for FP64 vectors; R <= 4 and R <= 8
 * use one pass of 4 or 8).  FP32 accumulation for FP32 and the narrow
 * types, FP64 multiply-adds for FP64 and single-double storage.
 * BF16 storage with 8 <= R <= 64 and A 16-byte aligned runs on the tensor
 * cores when the contraction is along the last mode (n_mode a multiple of
 * 8) or along another mode with v a multiple of 8 and v >= 64, and there are
 * at least as many 128-output tiles as SMs: X is split into three BF16
 * pieces (exact to binary32 precision; for mode 0 the slab scales are
 * folded into X first), every product of two BF16 values is exact, and the
 * MMAs accumulate in FP32.  FP32 storage with A 16-byte aligned runs on the
 * tensor cores as well, along the last mode (n_mode a multiple of 4,
 * 8 <= R <= 64) or along another mode (v a multiple of 4, v >= 32,
 * 8 < R <= 64), with the same tile condition: tf32 MMAs on A and its low
 * part A - trunc(A) against the two parts of X, with products dropped below
 * 2^-20 of |A X|.  The workspace
 * holds the pieces of X (tmc_workspace_size includes them).
 * slab_scales: as for tvc_ex.  workspace: tmc_workspace_size(...) bytes (0
 * when the output columns fill the GPU without splitting n_mode).
 * Errors: TVC_ERR_INVALID_ARG for a bad shape, mode, dtype, R < 1, a NULL
 * pointer or a misaligned A, X or Y; TVC_ERR_WORKSPACE when the workspace is
 * too small; nothing is launched then.
 */
tvc_status tmc(const void* A, int order, const int64_t* dims, int mode, const void* X, int64_t R, void* Y,
               tvc_dtype dtype, const float* slab_scales, double alpha, double beta, void* workspace,
               size_t ws_bytes, tvc_stream_t stream);
size_t tmc_workspace_size(int order, const int64_t* dims, int mode, int64_t R, tvc_dtype dtype);

/*
 * Khatri-Rao product (Section 1): out = U_0 (.) U_1 (.) ... (.) U_{count-1},
 * the columnwise Kronecker product of `count` matrices U_m (rows[m] x R,
 * row-major, device), out[(i_0, ..., i_{count-1})][r] = prod_m U_m[i_m][r]
 * with i_0 the most significant index of the row (prod rows[m] rows, R
 * columns, row-major).  vdtype: TVC_F64 or TVC_F32 for all matrices.
 * Errors: TVC_ERR_INVALID_ARG (count outside 1..TVC_MAX_ORDER, R < 1, a
 * NULL or misaligned pointer, sizes too large); nothing is launched then.
 */
tvc_status khatri_rao(const void* const* mats, int count, const int64_t* rows, int64_t R, void* out,
                      tvc_dtype vdtype, tvc_stream_t stream);

/*
 * Matricized tensor times Khatri-Rao product for mode k (the core of CP
 * alternating least squares, Section 1):
 *     M[i_k][r] = sum over all other indices of A[i_0..i_{d-1}] prod_{m != k} X_m[i_m][r].
 * factors: host array of `order` device pointers; factors[m] (m != mode) is
 * the n_m x R factor matrix X_m, row-major, FP64 for TVC_F64 / TVC_F32D and
 * FP32 otherwise; factors[mode] is not read (may be NULL; for order 1 the
 * array may be NULL).  M: n_mode x R, row-major, same type.  A is read
 * once: the larger side of mode k (the modes before it, or after it) is
 * contracted first by one tensor-matrix contraction (tmc) with the
 * transposed Khatri-Rao product of its factors, then the small result with
 * the other side's Khatri-Rao rows, in a fixed order.  slab_scales: as for
 * tvc_ex (folded into the Khatri-Rao rows).  workspace:
 * mttkrp_workspace_size(...) bytes, 256-byte aligned (it holds the two
 * Khatri-Rao products, the R x n_k x (smaller side) intermediate and the
 * contraction's own workspace).  Errors as for tmc; TVC_ERR_WORKSPACE when
 * the workspace is missing or too small.
 */
tvc_status mttkrp(const void* A, int order, const int64_t* dims, int mode, const void* const* factors, int64_t R,
                  void* M, tvc_dtype dtype, const float* slab_scales, void* workspace, size_t ws_bytes,
                  tvc_stream_t stream);
size_t mttkrp_workspace_size(int order, const int64_t* dims, int mode, int64_t R, tvc_dtype dtype);

/*
 * tvc_noalloc: the same contraction as tvc_ex() with alpha = 1, beta = 0,
 * for callers that cannot allocate device memory: plug-ins whose host
 * framework owns every device allocation through its own pool, and
 * real-time or certified deployments that forbid device allocation after
 * start-up.  The paper has no counterpart: this is an interface of this
 * library only.  The call still makes ordinary CUDA runtime calls (device
 * query, kernel launches, and on the first call a symbol lookup), so it
 * cannot be used where CUDA calls are not allowed at all (for instance
 * inside a host function queued on a stream).
 * It allocates nothing and needs no workspace: its scratch (the split
 * pieces of x for FP64 and the split-K partial sums) is a fixed array of
 * TVC_NOALLOC_SCRATCH_BYTES that is part of the library's device image, so
 * every GPU that loads the library holds that memory until the process
 * exits.  Contractions whose scratch need (tvc_workspace_size) is larger
 * are refused with TVC_ERR_WORKSPACE before anything is launched.
 * The first call on a device looks up the scratch's device address (one
 * cudaGetSymbolAddress with that device current); make that first call
 * before any stream capture.  All calls on a device share the one array,
 * whose contents persist from call to call; calls that can overlap on the
 * GPU (different streams without ordering) race on it and give wrong
 * results, so order them on one stream or with events.
 */
#define TVC_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
tvc_status tvc_noalloc(const void* A, int order, const int64_t* dims, int mode, const void* x, void* y,
                       tvc_dtype dtype, const float* slab_scales, tvc_stream_t stream);

/* -------------------------------------------------------------- adjoint */

/*
 * Adjoints of Y = A x_mode x (by differentiation of the Section 3
 * definition; the paper gives no passage for them).  With gy the gradient
 * of a loss with respect to Y (N/n_mode entries, the layout of y):
 *     gx[j]       = sum_{i,l} A[(i*n_k + j)*v + l] * gy[i*v + l]
 *     gA[(i*n_k+j)*v+l] = gy[i*v + l] * x[j] + beta_A * gA[...]
 * gx (n_mode entries) is computed when gx != NULL (needs A; narrow storage
 * uses its slab scales, i.e. gx is the gradient with respect to x of the
 * dequantised contraction); gA (N entries, FP64 for TVC_F64, FP32
 * otherwise: the gradient with respect to the dequantised values) is
 * written when gA != NULL (needs x; beta_A == 0 means gA is not read).
 * workspace: tvc_backward_workspace_size(...) bytes (for gx).  Results are
 * deterministic (fixed-order reductions).
 */
tvc_status tvc_backward(const void* A, int order, const int64_t* dims, int mode, const void* x, const void* gy,
                        void* gx, void* gA, tvc_dtype dtype, const float* slab_scales, double beta_A,
                        void* workspace, size_t ws_bytes, tvc_stream_t stream);
size_t tvc_backward_workspace_size(int order, const int64_t* dims, int mode, tvc_dtype dtype);

/* -------------------------------------------------------------- storage */

/*
 * Per-slab low-precision storage of an FP32 tensor (Section 5.5 uses low
 * precision as a storage format only; arithmetic is promoted).  One FP32
 * scale per slab A[i_0, ...] (n_0 scales):
 *   TVC_E4M3: scale = amax(slab)/448 (1 for an all-zero slab), code =
 *             E4M3(value/scale) rounded to nearest even, saturating to +-448.
 *   TVC_BF16: scale = 1, code = BF16(value) rounded to nearest even, or the
 *             upper half of the binary32 when truncate != 0 (the paper's
 *             truncating "brain" format).
 *   TVC_F16:  scale = 1, code = binary16(value) rounded to nearest even (the
 *             paper's half-single storage; values of magnitude >= 65520
 *             become infinity).
 * src: N floats; codes: N bytes (E4M3) or N uint16 (BF16, F16); scales: n_0
 * floats; status_out: 1 device int, set to TVC_ERR_NONFINITE when an E4M3
 * slab holds NaN or Inf (its codes are then meaningless) or when an F16 code
 * is infinite or NaN (overflow or a non-finite source; every code is still
 * written).  All device pointers.  workspace:
 * tvc_quantise_workspace_size(...) bytes.
 */
tvc_status tvc_quantise(const float* src, int order, const int64_t* dims, tvc_dtype dtype, void* codes,
                        float* scales, int truncate, int* status_out, void* workspace, size_t ws_bytes,
                        tvc_stream_t stream);
size_t tvc_quantise_workspace_size(int order, const int64_t* dims);

/* ----------------------------------------------------------------- HOPM */

/*
 * Higher-order power method (Section 3; three-buffer Algorithm 1 for one
 * process): Gauss-Seidel sweeps over j = 0..order-1 of
 *     z_j = A x_{m != j} x_m,   x_j = z_j / ||z_j||_2,
 * for at most `iters` sweeps.  x[m] (m < order) are device vectors of n_m
 * entries (FP64 for TVC_F64, FP32 otherwise) holding the start vectors on
 * entry and the result on exit; x[0] is not read (the first update
 * overwrites it).  lambda = ||z_{order-1}|| of the last sweep, which equals
 * A(x_0, ..., x_{order-1}) at the end of that sweep.
 * Stopping rule (the paper gives none): after sweep t >= 2, stop when
 * tol > 0 and |lambda_t - lambda_{t-1}| <= tol * lambda_t; tol = 0 runs all
 * sweeps.  The whole run is queued on `stream` without host synchronisation.
 * Device outputs (nullable): lambda_out (1 double), sweeps_out (1 int),
 * status_out (1 int: TVC_OK, TVC_ERR_ZERO_NORM or TVC_ERR_NONFINITE; on
 * either error the offending x_j keeps its previous value and the run
 * stops), lambda_hist (iters doubles: lambda of each completed sweep).
 * A is streamed twice per sweep.  order >= 2.  Workspace: at least
 * hopm_workspace_size(order, dims, dtype) bytes of device memory, 256-byte
 * aligned; it holds the run's state, so concurrent runs need separate ones.
 */
tvc_status hopm(const void* A, int order, const int64_t* dims, void* const* x, int iters, double tol,
                double* lambda_out, int* sweeps_out, int* status_out, double* lambda_hist, tvc_dtype dtype,
                const float* slab_scales, void* workspace, size_t ws_bytes, tvc_stream_t stream);

/* Bytes of workspace hopm needs (0 for invalid arguments). */
size_t hopm_workspace_size(int order, const int64_t* dims, tvc_dtype dtype);

/*
 * Jacobi HOPM (a variant of the power method, not the paper's Algorithm 1):
 * every z_j = A x_{m != j} x_m of a sweep is formed from the vectors of the
 * previous sweep, then every x_j <- z_j / ||z_j||; lambda = ||z_{d-1}|| of
 * the sweep.  Results differ from hopm() (Gauss-Seidel) except at a fixed
 * point.  A is read through two views per sweep: T = A x_{d-1} x_{d-1} and
 * z_{d-1} = A^T (x_0 (x) ... (x) x_{d-2}); every other z_j comes from the
 * small T.  Arguments, outputs, stopping rule and status as for hopm().
 * Workspace: hopm_jacobi_workspace_size(order, dims, dtype) bytes.
 */
tvc_status hopm_jacobi(const void* A, int order, const int64_t* dims, void* const* x, int iters, double tol,
                       double* lambda_out, int* sweeps_out, int* status_out, double* lambda_hist, tvc_dtype dtype,
                       const float* slab_scales, void* workspace, size_t ws_bytes, tvc_stream_t stream);
size_t hopm_jacobi_workspace_size(int order, const int64_t* dims, tvc_dtype dtype);

/*
 * Reverse-mode gradient of `iters` HOPM sweeps (fixed count: the run this
 * differentiates used tol = 0, or pass the sweep count it reported) started
 * from x0[m] (device, not modified).  Upstream gradients: gx_final[m]
 * (device vectors of n_m, for the final x_m; the array or any entry may be
 * NULL = zero) and g_lambda (device double, NULL = zero).  Outputs: gA (N
 * entries, written; FP64 for TVC_F64, FP32 otherwise, the gradient with
 * respect to the dequantised values for narrow storage) and gstart[m]
 * (nullable array/entries: gradients with respect to the start vectors;
 * that of x0[0] is zero since x0[0] is never read).
 * The iterates are recomputed, not stored: only the d vectors at the start
 * of each sweep are kept (iters * sum(n_m) numbers), and every sweep is
 * recomputed from them during the reverse pass.  Cost per sweep: the two
 * forward passes over A, one pass per update for A x_j gz, and one update
 * of gA.  Workspace: hopm_backward_workspace_size(order, dims, dtype, iters).
 */
tvc_status hopm_backward(const void* A, int order, const int64_t* dims, void* const* x0, int iters,
                         void* const* gx_final, const double* g_lambda, void* gA, void* const* gstart,
                         tvc_dtype dtype, const float* slab_scales, void* workspace, size_t ws_bytes,
                         tvc_stream_t stream);
size_t hopm_backward_workspace_size(int order, const int64_t* dims, tvc_dtype dtype, int iters);

/* -------------------------------------------------------------- batches */

/*
 * Many independent FP32 tensors of any order and shape in one persistent
 * launch (the paper's task-based overlap of many contractions, Section
 * 4.3, done as a device work queue): one descriptor per tensor; the work is
 * cut into items of about 2^20 elements (output ranges of the contraction,
 * row ranges of gx, slab/row rectangles of gA), largest tensors first, and
 * pulled by persistent blocks from an atomic counter.  (hopm_batched runs
 * one block per tensor.)
 * All pointers in a descriptor are device pointers, FP32, dense row-major.
 */
typedef struct {
  const float* A;
  int order;
  int mode;
  int64_t dims[TVC_MAX_ORDER];
  const float* x; /* n_mode entries (forward, and gA)                  */
  float* y;       /* N/n_mode entries: y = A x_mode x (NULL: skip)     */
  const float* gy; /* N/n_mode entries (adjoints)                       */
  float* gx;      /* n_mode: sum_{i,l} A[i,j,l] gy[i,l] (NULL: skip)   */
  float* gA;      /* N: gy (x) x along mode (NULL: skip)               */
} tvc_batch_desc;

typedef struct {
  const float* A;
  int order; /* >= 2 */
  int64_t dims[TVC_MAX_ORDER];
  float* x[TVC_MAX_ORDER]; /* start vectors in, result out (x[0] not read) */
  double* lambda_out;      /* 1 double (nullable): norm of the last update  */
  int* status_out;         /* 1 int (nullable): TVC_OK / ZERO_NORM / NONFINITE */
} hopm_batch_desc;

/* Reuse the descriptors uploaded by the previous call on this workspace
 * (same count): the call then issues one memset and one kernel and does
 * not synchronise, so it can be captured in a CUDA graph. */
#define TVC_BATCH_PREUPLOADED 1

/* Without TVC_BATCH_PREUPLOADED the call uploads the descriptors and waits
 * for that copy (the host array may be freed on return). */
tvc_status tvc_batched(const tvc_batch_desc* descs, int count, int flags, void* workspace, size_t ws_bytes,
                       tvc_stream_t stream);
size_t tvc_batched_workspace_size(const tvc_batch_desc* descs, int count);

/* Times the candidate block mappings (lanes per output) of the forward
 * contraction of rows v == 1 on the tensors of each such shape class of the
 * batch and keeps the fastest for later calls of tvc_batched / hopm_batched
 * in this process; synchronises the stream.
 * workspace: tvc_batched_workspace_size(descs, count) bytes; a batch
 * uploaded on it before must be uploaded again (call without
 * TVC_BATCH_PREUPLOADED). */
tvc_status tvc_batched_autotune(const tvc_batch_desc* descs, int count, void* workspace, size_t ws_bytes,
                                tvc_stream_t stream);

/* `iters` Gauss-Seidel HOPM sweeps (Section 3, Algorithm 1's schedule) on
 * every tensor of the batch, one block per tensor; FP64 norms. */
tvc_status hopm_batched(const hopm_batch_desc* descs, int count, int iters, int flags, void* workspace,
                        size_t ws_bytes, tvc_stream_t stream);
size_t hopm_batched_workspace_size(const hopm_batch_desc* descs, int count);

/* ------------------------------------------- 1D split over virtual ranks */

/*
 * The distributed algorithms of Section 3 (dTVC, Eq. 1 and Eq. 2; dHOPM_3,
 * Algorithm 1) on one GPU: the tensor is cut along one dimension s into
 * `parts` slabs, each held in its own dense buffer as a rank would hold it,
 * and every rank's work is launched on the same stream.  Where p processes
 * would exchange data, the ranks' results are combined on the device: a
 * fixed-order sum in place of the all-reduce, disjoint writes in place of
 * the gather.  At most TVC_MAX_PARTS ranks.
 */
#define TVC_MAX_PARTS 64

/* Slab boundaries of the 1D split of a dimension of n entries over p ranks
 * (Section 3.1, "optimal division"): chunk = ceil(n / p) rounded up to a
 * multiple of `quantum` (>= 1; the vector length in elements, 1 for none),
 * ranks = ceil(n / chunk) <= p, so p may be lowered (n = 4, p = 3 gives two
 * ranks of 2).  starts (p + 1 int64, host) receives 0 = starts[0] < ... <
 * starts[ranks] = n.  Returns the number of ranks, or -1 when n < 1, p < 1,
 * p > TVC_MAX_PARTS or quantum < 1.  Host only; launches nothing. */
int tvc_split_1d(int64_t n, int p, int64_t quantum, int64_t* starts);

/* Copies the slab [start, end) along dimension s between a dense tensor of
 * `dims` and a dense slab of dims with n_s replaced by end - start
 * (Section 3.1: for s > 0 the slab is prod(n_0 .. n_{s-1}) strided runs of
 * the tensor).  insert = 0: tensor -> slab (dst is the slab); insert = 1:
 * slab -> tensor (src is the slab; the rest of the tensor is untouched).
 * elem_bytes: bytes per element (1, 2, 4 or 8).  Device pointers, no
 * overlap; stream-ordered. */
tvc_status tvc_slab_copy(const void* src, void* dst, int order, const int64_t* dims, int s, int64_t start,
                         int64_t end, size_t elem_bytes, int insert, tvc_stream_t stream);

/*
 * Distributed TVC over `parts` virtual ranks (Section 3.1).  slabs[r] is
 * rank r's dense subtensor: dims with n_s replaced by starts[r+1] -
 * starts[r] (starts as from tvc_split_1d; starts[0] = 0, starts[parts] =
 * dims[s]).  x: n_mode entries (FP64 for TVC_F64, FP32 otherwise), the
 * same vector on every rank.
 *   mode != s (Eq. 1): y[r] (parts device outputs) receives rank r's output
 *     slab, alpha * slabs[r] x_mode x + beta * y[r]: the output dims with
 *     the s dimension cut to rank r's range.  No combination step.
 *   mode == s (Eq. 2): rank r contracts its slab with its part of x,
 *     x[starts[r] .. starts[r+1]), into a full-size partial (N / n_mode
 *     entries, in the workspace); y[0] receives alpha * (sum over r, in
 *     ascending order) + beta * y[0].
 * slab_scales: the n_0 per-slab scales of the global tensor for narrow
 * storage (rank r uses scales + starts[r] when s = 0).  Workspace:
 * dtvc_workspace_size(...) bytes.
 */
tvc_status dtvc(const void* const* slabs, int parts, const int64_t* starts, int order, const int64_t* dims, int s,
                int mode, const void* x, void* const* y, tvc_dtype dtype, const float* slab_scales, double alpha,
                double beta, void* workspace, size_t ws_bytes, tvc_stream_t stream);
size_t dtvc_workspace_size(int parts, const int64_t* starts, int order, const int64_t* dims, int s, int mode,
                           tvc_dtype dtype);

/*
 * Distributed three-buffer HOPM (dHOPM_3, Algorithm 1) over `parts` virtual
 * ranks: every rank keeps its own prefix cache W and intermediate buffers
 * and computes, for each external iteration j, its local contraction of
 * all modes but j (with x_s restricted to its range for j != s).  For
 * j != s the n_j-entry partial vectors are summed in ascending rank order
 * (the all-reduce; Eq. 2's sum deferred to the normalisation); for j = s
 * each rank writes its disjoint range of z_s (the gather).  Normalisation,
 * lambda, stopping rule, status and outputs as for hopm().  x: the global
 * vectors (device, order entries).  Workspace: dhopm_workspace_size(...).
 */
tvc_status dhopm(const void* const* slabs, int parts, const int64_t* starts, int order, const int64_t* dims, int s,
                 void* const* x, int iters, double tol, double* lambda_out, int* sweeps_out, int* status_out,
                 double* lambda_hist, tvc_dtype dtype, const float* slab_scales, void* workspace, size_t ws_bytes,
                 tvc_stream_t stream);
size_t dhopm_workspace_size(int parts, const int64_t* starts, int order, const int64_t* dims, int s,
                            tvc_dtype dtype);

/* Sticky device error of the staged (TMA-fed) kernels: every wait in them
 * is bounded, and a wait that gives up records a nonzero code (1: the copy
 * engine's producer waited for a free buffer, 2: a consumer waited for a
 * tile, 3: draining copies at exit; 11-14 the same for the tensor-core
 * tensor-matrix contraction: 11 producer, 12 MMA issuer, 13 drain, 14 the
 * epilogue's wait for the last MMAs; 21-23 the same three for the FP64
 * small-slab / short-row kernel, 31-33 for the narrow-storage slab kernel)
 * and lets the kernel finish (a kernel of the tensor-core path also
 * releases its tensor memory); its results are then invalid.  Synchronises the device; returns
 * TVC_ERR_TIMEOUT when a code is set (and clears it when clear != 0). */
tvc_status tvc_device_error(int* code_out, int clear);

/* Reads a device status word (the status_out / status argument of hopm,
 * hopm_jacobi, hopm_backward, tvc_quantise and the batched power methods):
 * waits for the work queued on `stream` before it (a stream-ordered copy,
 * then a synchronisation of that stream) and stores the word's value, a
 * tvc_status code, in *host_out.  It synchronises, so it must not be
 * called on a stream that is being captured: it then returns
 * TVC_ERR_INVALID_ARG without touching the stream (the capture stays
 * valid).  Returns TVC_ERR_INVALID_ARG for a NULL pointer, TVC_ERR_CUDA if
 * the copy fails, else TVC_OK (whatever the word holds). */
tvc_status tvc_read_status(const int* dev_status, int* host_out, tvc_stream_t stream);

/* Number of CUDA kernels this library has launched in this process (all
 * devices, all entry points).  Host-side counter, incremented per launch;
 * lets a caller count the kernels of a timed region. */
uint64_t tvc_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* TVC_GB300_H */
