// Host-side declarations shared by the translation units of the library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/tvc.h"

namespace tvcg {

// Matricized view of a d-order tensor for one mode (Section 3): the tensor
// is read as u x n_k x v, with n0 the size of the first mode (slab count).
struct Shape {
  int order = 0;
  int mode = 0;
  int64_t dims[TVC_MAX_ORDER] = {};
  int64_t N = 0, u = 0, nk = 0, v = 0, uv = 0, n0 = 0, upi0 = 1;
};

// Validates order/dims/mode and fills the view.  Returns TVC_OK or
// TVC_ERR_INVALID_ARG (order out of range, a size < 1, N >= 2^62).
tvc_status make_shape(int order, const int64_t* dims, int mode, Shape* s);
tvc_status check_dims(int order, const int64_t* dims, int64_t* N);

size_t elem_size(tvc_dtype dt);
size_t vec_size(tvc_dtype dt);  // 8 for F64, 4 otherwise
bool valid_dtype(int dt);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
inline bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Stream-ordered scratch for the entry points that do not take a workspace:
// cudaMallocFromPoolAsync on `st` from a library-owned pool of the current
// device (created on first use, memory kept reserved once freed), released
// with cudaFreeAsync on the same stream after the work that uses it.  Calls
// on different streams get different memory; under stream capture the pair
// becomes the graph's own allocation and free nodes.  bytes == 0 gives NULL.
tvc_status stream_scratch_alloc(size_t bytes, cudaStream_t st, void** out);
tvc_status stream_scratch_free(void* p, cudaStream_t st);

// cuTensorMapEncodeTiled, looked up once through the runtime (no link to the
// driver library); NULL when the driver does not offer it.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled();

// Number of SMs of the current device (cached per device).
int device_sms();

tvc_status cuda_status(cudaError_t e);

// Adds n to the process-wide launch counter (tvc_kernel_launches).
void count_launches(int n);

// Launches of the TVC kernels (tvc.cu), used by the HOPM and batched paths.
// done (nullable, device): every kernel of the launch returns at once when
// *done != 0 (work queued behind a converged power method).
tvc_status tvc_launch(const void* A, const Shape& s, const void* x, void* y, tvc_dtype dt,
                      const float* scales, double alpha, double beta, void* ws, size_t ws_bytes,
                      cudaStream_t stream, const int* done = nullptr);
size_t tvc_ws_bytes(const Shape& s, tvc_dtype dt, const void* A);

// 1D split over virtual ranks (split.cu).  check_split validates parts,
// starts and s against the tensor; slab_dims gives rank r's dims.
tvc_status check_split(int parts, const int64_t* starts, int order, const int64_t* dims, int s);
void slab_dims(int order, const int64_t* dims, int s, const int64_t* starts, int r, int64_t* out);
// Combination of the ranks' vectors on the device: gather = 0 sums the
// nparts vectors of n entries in ascending order (out = alpha*sum + beta*out);
// gather = 1 writes part r to out[offs[r] .. offs[r+1]).  vdt: TVC_F64 or
// TVC_F32 vectors.  done (nullable, device): skip when *done != 0.
tvc_status combine_parts(const void* const* parts, int nparts, const int64_t* offs, int64_t n, void* out,
                         tvc_dtype vdt, int gather, double alpha, double beta, cudaStream_t st,
                         const int* done);

// Tensor-matrix contraction on the tensor cores (tmc_tc.cu): BF16 storage
// (any mode; see tmc_tc_supported) and FP32 storage along the last mode,
// 8 <= R <= 64, A 16-byte aligned, enough 128-output tiles for the GPU (a16
// stands for the alignment of A when A is NULL, for the workspace query).
// Workspace: the pieces of X.
bool tmc_tc_supported(const Shape& s, int64_t R, tvc_dtype dt, const void* A, bool a16);
size_t tmc_tc_ws_bytes(const Shape& s, int64_t R, tvc_dtype dt);
tvc_status tmc_tc_launch_f32(const void* A, const Shape& s, const float* X, int64_t R, float* Y, double alpha,
                             double beta, void* ws, size_t ws_bytes, cudaStream_t st);
tvc_status tmc_tc_launch(const void* A, const Shape& s, const float* X, int64_t R, float* Y, const float* scales,
                         double alpha, double beta, void* ws, size_t ws_bytes, cudaStream_t st);
// Sticky error word of that kernel's bounded waits (cleared when clear != 0).
tvc_status tmc_tc_device_error(int* code_out, int clear);

// One pass over an R x C row-major matrix M (FP32, BF16, F16 or E4M3
// storage) for T = M x (scaled per slab: T[r] *= scales[r / upi0] when
// scales is given) and z = M^T w (dual.cu).  dual_supported says whether
// the shape and alignment fit; dual_ws_bytes covers every 16-byte aligned M.
bool dual_supported(int64_t R, int64_t C, tvc_dtype dt, const void* M);
size_t dual_ws_bytes(int64_t R, int64_t C, tvc_dtype dt, const void* M);
tvc_status dual_launch(const void* M, int64_t R, int64_t C, tvc_dtype dt, const float* x, const float* w,
                       const float* scales, int64_t upi0, float* T, float* z, void* ws, size_t ws_bytes,
                       cudaStream_t st, const int* done);

}  // namespace tvcg
