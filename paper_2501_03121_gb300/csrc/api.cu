// Host utilities of the C ABI: status strings, shape validation, the
// library-owned per-device workspace.
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
std::vector<std::pair<void*, size_t>> g_ws;  // per device id
std::vector<int> g_sms;
}  // namespace

void* library_workspace(size_t bytes, tvc_status* st) {
  *st = TVC_OK;
  if (bytes == 0) return nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    *st = TVC_ERR_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_ws_mu);
  if ((int)g_ws.size() <= dev) g_ws.resize(dev + 1, {nullptr, 0});
  auto& slot = g_ws[dev];
  if (slot.second < bytes) {
    if (slot.first) {
      // The old buffer may still be used by queued work on any stream.
      cudaDeviceSynchronize();
      cudaFree(slot.first);
      slot = {nullptr, 0};
    }
    size_t want = align_up(bytes, (size_t)1 << 20);
    void* p = nullptr;
    if (cudaMalloc(&p, want) != cudaSuccess) {
      cudaGetLastError();
      *st = TVC_ERR_CUDA;
      return nullptr;
    }
    slot = {p, want};
  }
  return slot.first;
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
  int v = 0;
  if (cudaMemcpyAsync(&v, dev_status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return TVC_ERR_CUDA;
  *host_out = v;
  return TVC_OK;
}
