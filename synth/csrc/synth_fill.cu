// Device-side fill of the seeded synthetic inputs: the same counter-based
// definitions as synth/__init__.py, bit for bit.  Every floating-point step
// uses an explicitly rounded intrinsic (__dadd_rn, __dmul_rn, ...) so that
// nothing is contracted into a fused multiply-add.  Holds none of the
// contraction's arithmetic: it only turns (seed, stream, index) into numbers.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

struct W4 {
  uint32_t w0, w1, w2, w3;
};

// Philox4x32-10 (Salmon et al., SC'11).
__device__ __forceinline__ W4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; r++) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return W4{c0, c1, c2, c3};
}

__device__ __forceinline__ W4 words(uint64_t seed, uint32_t sid, uint64_t idx, uint32_t word3) {
  return philox((uint32_t)idx, (uint32_t)(idx >> 32), sid, word3, (uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ __forceinline__ double u53(uint32_t lo, uint32_t hi) {
  const uint64_t m = ((uint64_t)hi << 21) | (uint64_t)(lo >> 11);
  return __dadd_rn(__dmul_rn((double)m, 0x1p-52), -1.0);
}

__device__ double ln_f64(double s) {
  int e;
  double m = frexp(s, &e);
  if (m < 0.7071067811865476) {
    m = __dmul_rn(m, 2.0);
    e -= 1;
  }
  const double t = __ddiv_rn(__dadd_rn(m, -1.0), __dadd_rn(m, 1.0));
  const double t2 = __dmul_rn(t, t);
  double acc = 1.0 / 23.0;
  for (int k = 10; k >= 0; k--) acc = __dadd_rn(__dmul_rn(acc, t2), 1.0 / (double)(2 * k + 1));
  return __dadd_rn(__dmul_rn((double)e, 0.6931471805599453), __dmul_rn(2.0, __dmul_rn(t, acc)));
}

__device__ double exp_f64(double t) {
  const double r = __ddiv_rn(t, 16.0);
  double fact = 6227020800.0;
  double acc = __ddiv_rn(1.0, fact);
  for (int k = 12; k >= 0; k--) {
    fact = __ddiv_rn(fact, (double)(k + 1));
    acc = __dadd_rn(__dmul_rn(acc, r), __ddiv_rn(1.0, fact));
  }
  for (int q = 0; q < 4; q++) acc = __dmul_rn(acc, acc);
  return acc;
}

__device__ double gaussian(uint64_t seed, uint32_t sid, uint64_t idx) {
  for (uint32_t a = 0; a < 32; a++) {
    const W4 w = words(seed, sid, idx, a);
    const double u = u53(w.w0, w.w1), v = u53(w.w2, w.w3);
    const double s = __dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v));
    if (s > 0.0 && s < 1.0) return __dmul_rn(u, __dsqrt_rn(__ddiv_rn(__dmul_rn(-2.0, ln_f64(s)), s)));
  }
  return 0.0;
}

__device__ double lognormal(uint64_t seed, uint32_t sid, uint64_t idx) {
  const double g = gaussian(seed, sid, idx);
  const W4 w = words(seed, sid, idx, 32u);
  return __dmul_rn(g, exp_f64(__dmul_rn(3.0, u53(w.w0, w.w1))));
}

enum Kind { K_U64 = 0, K_U32 = 1, K_GAUSS = 2, K_LOGNORMAL = 3, K_PLANTED = 4 };

struct Planted {
  int order;
  int64_t dims[16];
  const double* us[16];
};

__device__ double planted(uint64_t seed, const Planted& pl, uint64_t idx) {
  int64_t rem = (int64_t)idx;
  int64_t dig[16];
  for (int q = pl.order - 1; q >= 0; q--) {
    dig[q] = rem % pl.dims[q];
    rem /= pl.dims[q];
  }
  double acc = __dmul_rn(10.0, pl.us[0][dig[0]]);
  for (int q = 1; q < pl.order; q++) acc = __dmul_rn(acc, pl.us[q][dig[q]]);
  return __dadd_rn(acc, __dmul_rn(0.01, gaussian(seed, 20u, idx)));
}

template <class T>
__global__ void fill_kernel(T* out, int64_t n, int64_t offset, uint64_t seed, uint32_t sid, int kind, Planted pl) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t idx = (uint64_t)(offset + i);
    double v;
    if (kind == K_U64) {
      const W4 w = words(seed, sid, idx, 0u);
      v = u53(w.w0, w.w1);
    } else if (kind == K_U32) {
      const W4 w = words(seed, sid, idx, 0u);
      v = __dadd_rn(__dmul_rn((double)(w.w0 >> 8), 0x1p-23), -1.0);
    } else if (kind == K_GAUSS) {
      v = gaussian(seed, sid, idx);
    } else if (kind == K_LOGNORMAL) {
      v = lognormal(seed, sid, idx);
    } else {
      v = planted(seed, pl, idx);
    }
    if constexpr (sizeof(T) == 8)
      out[i] = v;
    else
      out[i] = __double2float_rn(v);
  }
}

}  // namespace

// out[i] = value of element (offset + i) of stream sid under seed, for
// i < n.  kind: 0 uniform[-1,1) 53-bit, 1 uniform[-1,1) 24-bit, 2 Gaussian,
// 3 Gaussian * exp(U[-3,3]), 4 planted rank-1 (order, dims, us: device
// pointers to the normalised factors, FP64).  f32 != 0 writes binary32
// (rounded to nearest), else binary64.  Returns a cudaError_t value.
extern "C" int synth_fill(void* out, int f32, int64_t n, int64_t offset, uint64_t seed, uint32_t sid, int kind,
                          int order, const int64_t* dims, const double* const* us, void* stream) {
  Planted pl{};
  if (kind == K_PLANTED) {
    if (order < 1 || order > 16) return (int)cudaErrorInvalidValue;
    pl.order = order;
    for (int q = 0; q < order; q++) {
      pl.dims[q] = dims[q];
      pl.us[q] = us[q];
    }
  }
  if (n <= 0) return 0;
  int dev = 0, sms = 132;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n + 255) / 256;
  const int blocks = (int)(want < (int64_t)sms * 32 ? want : (int64_t)sms * 32);
  cudaStream_t st = (cudaStream_t)stream;
  if (f32)
    fill_kernel<float><<<blocks, 256, 0, st>>>((float*)out, n, offset, seed, sid, kind, pl);
  else
    fill_kernel<double><<<blocks, 256, 0, st>>>((double*)out, n, offset, seed, sid, kind, pl);
  return (int)cudaGetLastError();
}
