// Per-slab low-precision storage of an FP32 tensor (the storage-only use of
// low precision of Section 5.5): one FP32 scale per slab A[i_0, ...].
//   E4M3: scale = amax(slab) / 448 (1 when the slab is all zero); code =
//         E4M3(value / scale), round to nearest even, saturating at +-448
//         (OCP "satfinite"), NaN -> 0x7F.
//   BF16: scale = 1; code = BF16(value), round to nearest even, or the upper
//         half of the binary32 when truncation is asked for (the paper's
//         "brain" conversion); NaN -> 0x7FC0 with the input's sign.
//   F16:  scale = 1; code = binary16(value), round to nearest even (the
//         paper's half-single storage), overflow to infinity; NaN -> 0x7E00
//         with the input's sign; an infinite or NaN code sets the status.
// The slab maximum is an order-independent reduction (integer max of the
// non-negative binary32 bit patterns), so the codes are deterministic.
#include "common.cuh"
#include "internal.h"

namespace tvcg {

// amax bits per slab; NaN maps above every finite value (0x7FC00000 > inf).
__global__ void quant_amax_kernel(const float* __restrict__ src, int64_t n0, int64_t slab, unsigned* amax) {
  const int64_t per = (slab + gridDim.y - 1) / gridDim.y;
  for (int64_t i = blockIdx.x; i < n0; i += gridDim.x) {
    const int64_t lo = (int64_t)blockIdx.y * per, hi = min(slab, lo + per);
    unsigned m = 0;
    for (int64_t f = lo + threadIdx.x; f < hi; f += blockDim.x) {
      unsigned b = __float_as_uint(src[i * slab + f]) & 0x7FFFFFFFu;
      if (b > 0x7F800000u) b = 0x7FC00000u;
      m = max(m, b);
    }
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(amax + i, m);
  }
}

__global__ void quant_scale_kernel(const unsigned* amax, float* scales, int64_t n0, int e4m3, int* status) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n0; i += (int64_t)gridDim.x * blockDim.x) {
    float sc = 1.0f;
    if (e4m3) {
      const unsigned b = amax[i];
      if (b >= 0x7F800000u) {
        atomicExch(status, (int)TVC_ERR_NONFINITE);
      } else if (b != 0u) {
        sc = __fdiv_rn(__uint_as_float(b), 448.0f);
      }
    }
    scales[i] = sc;
  }
}

enum QuantFmt { Q_BF16 = 0, Q_E4M3 = 1, Q_F16 = 2 };

__global__ void quant_codes_kernel(const float* __restrict__ src, int64_t N, int64_t slab, const float* scales,
                                   void* codes, int fmt, int truncate, int* status) {
  int nonfinite = 0;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < N; f += (int64_t)gridDim.x * blockDim.x) {
    const float v = src[f];
    if (fmt == Q_F16) {
      uint16_t c;
      if (isnan(v)) {
        c = (uint16_t)(((__float_as_uint(v) >> 16) & 0x8000u) | 0x7E00u);
      } else {
        const __half h = __float2half_rn(v);
        c = __half_as_ushort(h);
      }
      nonfinite |= ((c & 0x7C00u) == 0x7C00u);
      static_cast<uint16_t*>(codes)[f] = c;
    } else if (fmt == Q_E4M3) {
      const float q = __fdiv_rn(v, scales[f / slab]);
      static_cast<uint8_t*>(codes)[f] = (uint8_t)__nv_cvt_float_to_fp8(q, __NV_SATFINITE, __NV_E4M3);
    } else {
      uint16_t c;
      const unsigned b = __float_as_uint(v);
      if (isnan(v)) {
        c = (uint16_t)(((b >> 16) & 0x8000u) | 0x7FC0u);
      } else if (truncate) {
        c = (uint16_t)(b >> 16);
      } else {
        __nv_bfloat16 h = __float2bfloat16_rn(v);
        c = *reinterpret_cast<uint16_t*>(&h);
      }
      static_cast<uint16_t*>(codes)[f] = c;
    }
  }
  if (nonfinite) atomicExch(status, (int)TVC_ERR_NONFINITE);
}

}  // namespace tvcg

using namespace tvcg;

extern "C" size_t tvc_quantise_workspace_size(int order, const int64_t* dims) {
  if (check_dims(order, dims, nullptr) != TVC_OK) return 0;
  return align_up((size_t)dims[0] * sizeof(unsigned), 256) + 256;
}

extern "C" tvc_status tvc_quantise(const float* src, int order, const int64_t* dims, tvc_dtype dtype, void* codes,
                                   float* scales, int truncate, int* status_out, void* workspace, size_t ws_bytes,
                                   tvc_stream_t stream) {
  int64_t N;
  if (check_dims(order, dims, &N) != TVC_OK) return TVC_ERR_INVALID_ARG;
  if ((dtype != TVC_BF16 && dtype != TVC_E4M3 && dtype != TVC_F16) || !src || !codes || !scales || !status_out)
    return TVC_ERR_INVALID_ARG;
  if (!aligned(src, 4) || !aligned(scales, 4) || !aligned(codes, elem_size(dtype))) return TVC_ERR_INVALID_ARG;
  if (!workspace || ws_bytes < tvc_quantise_workspace_size(order, dims)) return TVC_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n0 = dims[0], slab = N / n0;
  unsigned* amax = static_cast<unsigned*>(workspace);
  const int e4m3 = dtype == TVC_E4M3;
  cudaMemsetAsync(status_out, 0, sizeof(int), st);
  int launches = 0;
  if (e4m3) {
    cudaMemsetAsync(amax, 0, (size_t)n0 * sizeof(unsigned), st);
    const int64_t by = std::min<int64_t>(64, std::max<int64_t>(1, slab / (1 << 16)));
    dim3 grid((unsigned)std::min<int64_t>(n0, 65535), (unsigned)by);
    quant_amax_kernel<<<grid, 256, 0, st>>>(src, n0, slab, amax);
    launches++;
  }
  quant_scale_kernel<<<(unsigned)std::min<int64_t>((n0 + 255) / 256, 4096), 256, 0, st>>>(amax, scales, n0, e4m3,
                                                                                         status_out);
  const int blocks = (int)std::min<int64_t>((N + 255) / 256, (int64_t)device_sms() * 32);
  const int fmt = e4m3 ? Q_E4M3 : (dtype == TVC_F16 ? Q_F16 : Q_BF16);
  quant_codes_kernel<<<blocks, 256, 0, st>>>(src, N, slab, scales, codes, fmt, truncate, status_out);
  count_launches(launches + 2);
  return cuda_status(cudaGetLastError());
}
