// tvc_noalloc: the contraction of tvc()/tvc_ex() for callers that must not
// allocate device memory.  Two kinds of caller cannot call cudaMalloc:
// plug-ins whose host framework owns every device allocation through its own
// pool (an allocation behind its back is invisible to its accounting and can
// push it out of memory), and real-time or certified deployments that forbid
// device allocation once start-up is over (an allocation can block on the
// driver and its failure mode is hard to bound).  tvc() allocates its
// scratch per call and tvc_ex() needs a workspace from the caller, so this
// entry point instead uses a fixed scratch array that is part of the
// library's device image.  It still makes ordinary CUDA runtime calls
// (device query, symbol lookup on first use, kernel launches), so it is no
// use where CUDA calls are forbidden altogether.
#include <mutex>

#include "internal.h"

namespace tvcg {
namespace {

// The scratch: split pieces of x (FP64) and split-K partial sums.  Every GPU
// that loads the library holds these bytes until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TVC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device.  Host code may not
// use g_noalloc_scratch itself (on the host that name is only a stand-in),
// so the address is looked up once per device, with that device current.
tvc_status scratch_on_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return TVC_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return TVC_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return TVC_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return TVC_OK;
}

}  // namespace
}  // namespace tvcg

using namespace tvcg;

extern "C" tvc_status tvc_noalloc(const void* A, int order, const int64_t* dims, int mode, const void* x, void* y,
                                  tvc_dtype dtype, const float* slab_scales, tvc_stream_t stream) {
  if (!valid_dtype(dtype)) return TVC_ERR_INVALID_ARG;
  Shape s;
  tvc_status st = make_shape(order, dims, mode, &s);
  if (st != TVC_OK) return st;
  if (!A || !x || !y) return TVC_ERR_INVALID_ARG;
  const size_t es = elem_size(dtype), vs = vec_size(dtype);
  if (!aligned(A, es) || !aligned(x, vs) || !aligned(y, vs)) return TVC_ERR_INVALID_ARG;
  // Size check before any CUDA call: too large a contraction is refused.
  const size_t need = tvc_ws_bytes(s, dtype, A);
  if (need > (size_t)TVC_NOALLOC_SCRATCH_BYTES) return TVC_ERR_WORKSPACE;
  void* scratch = nullptr;
  st = scratch_on_current_device(&scratch);
  if (st != TVC_OK) return st;
  // Nothing in the scratch needs to start at zero: the kernels write every
  // byte they later read (split x, then the partial sums) within the call.
  return tvc_launch(A, s, x, y, dtype, slab_scales, 1.0, 0.0, scratch, (size_t)TVC_NOALLOC_SCRATCH_BYTES,
                    (cudaStream_t)stream);
}
