// The 1D split of Section 3.1 over virtual ranks on one GPU: the "optimal
// division" of a dimension, slab copies between a tensor and its ranks'
// dense subtensors, the distributed TVC (Eq. 1: disjoint output slabs,
// Eq. 2: full-size partials summed), and the device-side combination step
// (fixed-order sum for the all-reduce, disjoint writes for the gather) that
// the distributed HOPM (hopm.cu) shares.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace tvcg {

namespace {

__device__ __forceinline__ bool split_skip(const int* done) {
  return done != nullptr && *reinterpret_cast<const volatile int*>(done) != 0;
}

// Copies w runs of `run` units from src (pitch sp) to dst (pitch dp).
template <class U>
__global__ void slab_copy_kernel(const U* __restrict__ src, U* __restrict__ dst, int64_t w, int64_t run, int64_t sp,
                                 int64_t dp) {
  for (int64_t a = blockIdx.y; a < w; a += gridDim.y) {
    const U* s = src + a * sp;
    U* d = dst + a * dp;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < run; b += (int64_t)gridDim.x * blockDim.x)
      d[b] = s[b];
  }
}

struct PartsArgs {
  int nparts;
  const void* p[TVC_MAX_PARTS];
  int64_t off[TVC_MAX_PARTS + 1];
};

// out[o] = alpha * sum_r part_r[o] (r ascending) + beta * out[o].
template <class V>
__global__ void combine_sum_kernel(const PartsArgs pa, V* __restrict__ out, int64_t n, double alpha, double beta,
                                   const int* done) {
  if (split_skip(done)) return;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
    V r;
    if constexpr (sizeof(V) == 8) {
      double s = 0.0;
      for (int q = 0; q < pa.nparts; q++) s += static_cast<const double*>(pa.p[q])[o];
      r = alpha * s;
      if (beta != 0.0) r += beta * out[o];
    } else {
      KahanF32 s;
      for (int q = 0; q < pa.nparts; q++) s.add(static_cast<const float*>(pa.p[q])[o]);
      r = (float)alpha * s.value();
      if (beta != 0.0) r += (float)beta * out[o];
    }
    out[o] = r;
  }
}

// out[off[r] + i] = part_r[i] for i < off[r+1] - off[r]; blockIdx.y = r.
template <class V>
__global__ void combine_gather_kernel(const PartsArgs pa, V* __restrict__ out, const int* done) {
  if (split_skip(done)) return;
  const int r = blockIdx.y;
  const int64_t len = pa.off[r + 1] - pa.off[r];
  const V* src = static_cast<const V*>(pa.p[r]);
  V* dst = out + pa.off[r];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

tvc_status check_split(int parts, const int64_t* starts, int order, const int64_t* dims, int s) {
  int64_t N = 0;
  if (check_dims(order, dims, &N) != TVC_OK) return TVC_ERR_INVALID_ARG;
  if (parts < 1 || parts > TVC_MAX_PARTS || starts == nullptr || s < 0 || s >= order) return TVC_ERR_INVALID_ARG;
  if (starts[0] != 0 || starts[parts] != dims[s]) return TVC_ERR_INVALID_ARG;
  for (int r = 0; r < parts; r++)
    if (starts[r + 1] <= starts[r]) return TVC_ERR_INVALID_ARG;
  return TVC_OK;
}

void slab_dims(int order, const int64_t* dims, int s, const int64_t* starts, int r, int64_t* out) {
  for (int i = 0; i < order; i++) out[i] = dims[i];
  out[s] = starts[r + 1] - starts[r];
}

tvc_status combine_parts(const void* const* parts, int nparts, const int64_t* offs, int64_t n, void* out,
                         tvc_dtype vdt, int gather, double alpha, double beta, cudaStream_t st, const int* done) {
  if (nparts < 1 || nparts > TVC_MAX_PARTS) return TVC_ERR_INVALID_ARG;
  PartsArgs pa{};
  pa.nparts = nparts;
  for (int r = 0; r < nparts; r++) pa.p[r] = parts[r];
  if (gather) {
    int64_t longest = 1;
    for (int r = 0; r <= nparts; r++) pa.off[r] = offs[r];
    for (int r = 0; r < nparts; r++) longest = std::max<int64_t>(longest, offs[r + 1] - offs[r]);
    const dim3 grid((unsigned)std::min<int64_t>(ceil_div64(longest, 256), 1024), (unsigned)nparts);
    if (vdt == TVC_F64)
      combine_gather_kernel<double><<<grid, 256, 0, st>>>(pa, static_cast<double*>(out), done);
    else
      combine_gather_kernel<float><<<grid, 256, 0, st>>>(pa, static_cast<float*>(out), done);
  } else {
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div64(n, 256), 8192));
    if (vdt == TVC_F64)
      combine_sum_kernel<double><<<blocks, 256, 0, st>>>(pa, static_cast<double*>(out), n, alpha, beta, done);
    else
      combine_sum_kernel<float><<<blocks, 256, 0, st>>>(pa, static_cast<float*>(out), n, alpha, beta, done);
  }
  count_launches(1);
  return cuda_status(cudaGetLastError());
}

}  // namespace tvcg

using namespace tvcg;

extern "C" int tvc_split_1d(int64_t n, int p, int64_t quantum, int64_t* starts) {
  if (n < 1 || p < 1 || p > TVC_MAX_PARTS || quantum < 1 || starts == nullptr) return -1;
  int64_t chunk = ceil_div64(n, p);
  chunk = ceil_div64(chunk, quantum) * quantum;
  const int ranks = (int)ceil_div64(n, chunk);
  for (int r = 0; r < ranks; r++) starts[r] = (int64_t)r * chunk;
  starts[ranks] = n;
  return ranks;
}

extern "C" tvc_status tvc_slab_copy(const void* src, void* dst, int order, const int64_t* dims, int s, int64_t start,
                                    int64_t end, size_t elem_bytes, int insert, tvc_stream_t stream) {
  int64_t N = 0;
  if (check_dims(order, dims, &N) != TVC_OK || s < 0 || s >= order) return TVC_ERR_INVALID_ARG;
  if (!(elem_bytes == 1 || elem_bytes == 2 || elem_bytes == 4 || elem_bytes == 8)) return TVC_ERR_INVALID_ARG;
  if (start < 0 || end <= start || end > dims[s] || src == nullptr || dst == nullptr) return TVC_ERR_INVALID_ARG;
  int64_t w = 1, tail = 1;
  for (int i = 0; i < s; i++) w *= dims[i];
  for (int i = s + 1; i < order; i++) tail *= dims[i];
  const int64_t es = (int64_t)elem_bytes;
  const int64_t run_b = (end - start) * tail * es;
  const int64_t full_b = dims[s] * tail * es;
  const char* sb = static_cast<const char*>(src);
  char* db = static_cast<char*>(dst);
  int64_t sp_b, dp_b;
  if (insert) {
    db += start * tail * es;
    sp_b = run_b;
    dp_b = full_b;
  } else {
    sb += start * tail * es;
    sp_b = full_b;
    dp_b = run_b;
  }
  // widest unit that divides every extent and both start addresses
  int64_t g = 16;
  while (g > 1 && (run_b % g || sp_b % g || dp_b % g || (uintptr_t)sb % g || (uintptr_t)db % g)) g >>= 1;
  const int64_t run = run_b / g, sp = sp_b / g, dp = dp_b / g;
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div64(run, 256), 1024));
  const unsigned gy = (unsigned)std::max<int64_t>(1, std::min<int64_t>(w, std::max<int64_t>(1, 65535 / gx)));
  const dim3 grid(gx, gy);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  switch (g) {
    case 16:
      slab_copy_kernel<uint4><<<grid, 256, 0, st>>>(reinterpret_cast<const uint4*>(sb), reinterpret_cast<uint4*>(db),
                                                    w, run, sp, dp);
      break;
    case 8:
      slab_copy_kernel<uint2><<<grid, 256, 0, st>>>(reinterpret_cast<const uint2*>(sb), reinterpret_cast<uint2*>(db),
                                                    w, run, sp, dp);
      break;
    case 4:
      slab_copy_kernel<uint32_t><<<grid, 256, 0, st>>>(reinterpret_cast<const uint32_t*>(sb),
                                                       reinterpret_cast<uint32_t*>(db), w, run, sp, dp);
      break;
    case 2:
      slab_copy_kernel<uint16_t><<<grid, 256, 0, st>>>(reinterpret_cast<const uint16_t*>(sb),
                                                       reinterpret_cast<uint16_t*>(db), w, run, sp, dp);
      break;
    default:
      slab_copy_kernel<uint8_t><<<grid, 256, 0, st>>>(reinterpret_cast<const uint8_t*>(sb),
                                                      reinterpret_cast<uint8_t*>(db), w, run, sp, dp);
      break;
  }
  count_launches(1);
  return cuda_status(cudaGetLastError());
}

namespace {

// TVC workspace of the largest rank (any slab alignment) and, for mode == s,
// the ranks' full-size partials after it.
struct DtvcLayout {
  size_t tvc = 0, off_partials = 0, partial_bytes = 0, total = 0;
};

DtvcLayout dtvc_layout(int parts, const int64_t* starts, int order, const int64_t* dims, int s, int mode,
                       tvc_dtype dt) {
  DtvcLayout L;
  int64_t dr[TVC_MAX_ORDER];
  for (int r = 0; r < parts; r++) {
    slab_dims(order, dims, s, starts, r, dr);
    Shape sh;
    make_shape(order, dr, mode, &sh);
    for (uintptr_t al = elem_size(dt); al <= 256; al *= 2)
      L.tvc = std::max(L.tvc, tvc_ws_bytes(sh, dt, reinterpret_cast<const void*>(al)));
  }
  L.off_partials = align_up(L.tvc, 256);
  L.total = L.off_partials;
  if (mode == s) {
    int64_t N = 1;
    for (int i = 0; i < order; i++) N *= dims[i];
    L.partial_bytes = align_up((size_t)(N / dims[mode]) * vec_size(dt), 256);
    L.total += (size_t)parts * L.partial_bytes;
  }
  return L;
}

}  // namespace

extern "C" size_t dtvc_workspace_size(int parts, const int64_t* starts, int order, const int64_t* dims, int s,
                                      int mode, tvc_dtype dtype) {
  if (!valid_dtype(dtype) || check_split(parts, starts, order, dims, s) != TVC_OK || mode < 0 || mode >= order)
    return 0;
  return dtvc_layout(parts, starts, order, dims, s, mode, dtype).total;
}

extern "C" tvc_status dtvc(const void* const* slabs, int parts, const int64_t* starts, int order, const int64_t* dims,
                           int s, int mode, const void* x, void* const* y, tvc_dtype dtype, const float* slab_scales,
                           double alpha, double beta, void* workspace, size_t ws_bytes, tvc_stream_t stream) {
  if (!valid_dtype(dtype) || check_split(parts, starts, order, dims, s) != TVC_OK) return TVC_ERR_INVALID_ARG;
  if (mode < 0 || mode >= order || slabs == nullptr || x == nullptr || y == nullptr) return TVC_ERR_INVALID_ARG;
  const int nout = (mode == s) ? 1 : parts;
  for (int r = 0; r < parts; r++)
    if (slabs[r] == nullptr) return TVC_ERR_INVALID_ARG;
  for (int r = 0; r < nout; r++)
    if (y[r] == nullptr) return TVC_ERR_INVALID_ARG;
  const DtvcLayout L = dtvc_layout(parts, starts, order, dims, s, mode, dtype);
  if (L.total > 0 && (workspace == nullptr || ws_bytes < L.total)) return TVC_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(workspace);
  const size_t vs = vec_size(dtype);
  int64_t dr[TVC_MAX_ORDER];
  const void* partial[TVC_MAX_PARTS];
  for (int r = 0; r < parts; r++) {
    slab_dims(order, dims, s, starts, r, dr);
    Shape sh;
    if (make_shape(order, dr, mode, &sh) != TVC_OK) return TVC_ERR_INVALID_ARG;
    const float* sc = slab_scales ? slab_scales + (s == 0 ? starts[r] : 0) : nullptr;
    tvc_status rc;
    if (mode == s) {
      // Eq. 2: rank r's part of x, a full-size partial, summed below.
      const void* xr = static_cast<const char*>(x) + (size_t)starts[r] * vs;
      void* pr = w + L.off_partials + (size_t)r * L.partial_bytes;
      partial[r] = pr;
      rc = tvc_launch(slabs[r], sh, xr, pr, dtype, sc, 1.0, 0.0, w, L.tvc, st);
    } else {
      // Eq. 1: disjoint output slabs, no exchange.
      rc = tvc_launch(slabs[r], sh, x, y[r], dtype, sc, alpha, beta, w, L.tvc, st);
    }
    if (rc != TVC_OK) return rc;
  }
  if (mode == s) {
    int64_t N = 1;
    for (int i = 0; i < order; i++) N *= dims[i];
    return combine_parts(partial, parts, nullptr, N / dims[mode], y[0], vec_size(dtype) == 8 ? TVC_F64 : TVC_F32, 0,
                         alpha, beta, st, nullptr);
  }
  return TVC_OK;
}
