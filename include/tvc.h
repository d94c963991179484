/*
 * tvc.h -- C ABI of the GB300 tensor-vector contraction library.
 *
 * Method: Martinez-Ferrer, Yzelman, Beltran, "Distributed and heterogeneous
 * tensor-vector contraction algorithms for high performance computing"
 * (arXiv 2501.03121).  This library is the single-GPU hot path of that
 * method: the mode-oblivious dense tensor-vector contraction (TVC) and the
 * higher-order power method (HOPM) built on it, with low-precision storage,
 * adjoints and batching.
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
 *   prefix tensors) are FP64 for TVC_F64 and FP32 for every other type.
 *   TVC_BF16 and TVC_E4M3 carry one FP32 scale per slab A[i_0, ...]
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
 *   different workspaces.
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
  TVC_E4M3 = 3  /* OCP FP8 E4M3 (bias 7, max 448), per-slab FP32 scale   */
} tvc_dtype;

typedef enum {
  TVC_OK = 0,
  TVC_ERR_INVALID_ARG = 1, /* bad pointer, order, size, mode or dtype         */
  TVC_ERR_UNSUPPORTED = 2, /* valid but not supported by this build           */
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
 * Uses a workspace the library allocates once per device when the shape
 * needs one (see tvc_ex to pass your own).  Narrow types use unit scales.
 */
tvc_status tvc(const void* A, int order, const int64_t* dims, int mode, const void* x, void* y,
               tvc_dtype dtype, tvc_stream_t stream);

/*
 * Y := alpha * (A x_mode x) + beta * Y  (the BLAS-like form of Eq. 1 for a
 * single process).  beta == 0 means y is not read (NaN in y is ignored).
 * slab_scales: n_0 FP32 scales for TVC_BF16 / TVC_E4M3, ignored otherwise.
 * workspace: device memory of at least tvc_workspace_size(...) bytes; it
 * may be NULL when that size is 0.  Returns TVC_ERR_WORKSPACE if too small.
 */
tvc_status tvc_ex(const void* A, int order, const int64_t* dims, int mode, const void* x, void* y,
                  tvc_dtype dtype, const float* slab_scales, double alpha, double beta,
                  void* workspace, size_t ws_bytes, tvc_stream_t stream);

/* Bytes of workspace tvc_ex needs for this shape (0 when none); the same
 * plan is used by tvc_ex for the same arguments on the same device. */
size_t tvc_workspace_size(int order, const int64_t* dims, int mode, tvc_dtype dtype);

/* Number of CUDA kernels this library has launched in this process (all
 * devices, all entry points).  Host-side counter, incremented per launch;
 * lets a caller count the kernels of a timed region. */
uint64_t tvc_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* TVC_GB300_H */
