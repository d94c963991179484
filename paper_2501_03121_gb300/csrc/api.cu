// Host utilities of the C ABI: status strings, shape validation, the
// library-owned stream-ordered memory pool of tvc().
#include <atomic>
#include <mutex>
#include <vector>

#include "internal.h"

namespace tvcg {

tvc_status check_dims(int order, const int64_t* dims, int64_t* N) {
  if (order < 1 || order > TVC_MAX_ORDER || dims == nullptr) return TVC_ERR_INVALID_ARG;
  int64_t n = 1;
  for (int i = 0; i < order; i++) {
    if (dims[i] < 1) return TVC_ERR_INVALID_ARG;
    int64_t m;
    if (__builtin_mul_overflow(n, dims[i], &m) || m >= ((int64_t)1 << 62)) return TVC_ERR_INVALID_ARG;
    n = m;
  }
  if (N) *N = n;
  return TVC_OK;
}

tvc_status make_shape(int order, const int64_t* dims, int mode, Shape* s) {
  int64_t N;
  tvc_status st = check_dims(order, dims, &N);
  if (st != TVC_OK) return st;
  if (mode < 0 || mode >= order) return TVC_ERR_INVALID_ARG;
  s->order = order;
  s->mode = mode;
  for (int i = 0; i < order; i++) s->dims[i] = dims[i];
  s->N = N;
  s->u = 1;
  for (int i = 0; i < mode; i++) s->u *= dims[i];
  s->nk = dims[mode];
  s->v = 1;
  for (int i = mode + 1; i < order; i++) s->v *= dims[i];
  s->uv = s->u * s->v;
  s->n0 = dims[0];
  // Output row i (of u) lies in slab i / upi0 when mode > 0.
  s->upi0 = (mode > 0) ? s->u / dims[0] : 1;
  return TVC_OK;
}

bool valid_dtype(int dt) { return dt >= TVC_F64 && dt <= TVC_F32D; }

size_t elem_size(tvc_dtype dt) {
  switch (dt) {
    case TVC_F64: return 8;
    case TVC_F32: return 4;
    case TVC_BF16: return 2;
    case TVC_E4M3: return 1;
    case TVC_F16: return 2;
    case TVC_F32D: return 4;
  }
  return 0;
}

size_t vec_size(tvc_dtype dt) { return (dt == TVC_F64 || dt == TVC_F32D) ? 8 : 4; }

tvc_status cuda_status(cudaError_t e) { return e == cudaSuccess ? TVC_OK : TVC_ERR_CUDA; }

static std::atomic<uint64_t> g_launches{0};
void count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

namespace {
std::mutex g_ws_mu;
std::vector<cudaMemPool_t> g_pools;  // per device id
std::vector<int> g_sms;
}  // namespace

// The library's stream-ordered memory pool on the current device, created on
// first use.  Its release threshold is "never", so memory freed back to it
// stays reserved and later allocations of the same size cost no driver
// mapping.
static tvc_status device_pool(cudaMemPool_t* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return TVC_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_ws_mu);
  if ((int)g_pools.size() <= dev) g_pools.resize(dev + 1, nullptr);
  if (g_pools[dev] == nullptr) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return TVC_ERR_CUDA;
    }
    uint64_t keep = ~(uint64_t)0;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = pool;
  }
  *out = g_pools[dev];
  return TVC_OK;
}

tvc_status stream_scratch_alloc(size_t bytes, cudaStream_t st, void** out) {
  *out = nullptr;
  if (bytes == 0) return TVC_OK;
  cudaMemPool_t pool = nullptr;
  tvc_status s = device_pool(&pool);
  if (s != TVC_OK) return s;
  if (cudaMallocFromPoolAsync(out, bytes, pool, st) != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
    return TVC_ERR_CUDA;
  }
  return TVC_OK;
}

tvc_status stream_scratch_free(void* p, cudaStream_t st) {
  if (p == nullptr) return TVC_OK;
  return cuda_status(cudaFreeAsync(p, st));
}

int device_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  std::lock_guard<std::mutex> lk(g_ws_mu);
  if ((int)g_sms.size() <= dev) g_sms.resize(dev + 1, 0);
  if (g_sms[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    g_sms[dev] = n;
  }
  return g_sms[dev];
}

}  // namespace tvcg

extern "C" uint64_t tvc_kernel_launches(void) { return tvcg::g_launches.load(); }

extern "C" const char* tvc_status_string(tvc_status s) {
  switch (s) {
    case TVC_OK: return "TVC_OK";
    case TVC_ERR_INVALID_ARG: return "TVC_ERR_INVALID_ARG: bad pointer, order, size, mode or dtype";
    case TVC_ERR_UNSUPPORTED: return "TVC_ERR_UNSUPPORTED: not supported by this library";
    case TVC_ERR_WORKSPACE: return "TVC_ERR_WORKSPACE: workspace too small";
    case TVC_ERR_CUDA: return "TVC_ERR_CUDA: a CUDA call failed";
    case TVC_ERR_ZERO_NORM: return "TVC_ERR_ZERO_NORM: an update vector had zero norm";
    case TVC_ERR_NONFINITE: return "TVC_ERR_NONFINITE: NaN or Inf met in a norm";
    case TVC_ERR_TIMEOUT: return "TVC_ERR_TIMEOUT: a bounded device wait gave up";
  }
  return "unknown tvc_status";
}

extern "C" tvc_status tvc_read_status(const int* dev_status, int* host_out, tvc_stream_t stream) {
  if (!dev_status || !host_out) return TVC_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // The read waits for the stream, which a stream being captured cannot do:
  // refuse before touching it, so that the capture stays valid.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    return TVC_ERR_CUDA;
  }
  if (cap != cudaStreamCaptureStatusNone) return TVC_ERR_INVALID_ARG;
  int v = 0;
  if (cudaMemcpyAsync(&v, dev_status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return TVC_ERR_CUDA;
  *host_out = v;
  return TVC_OK;
}
