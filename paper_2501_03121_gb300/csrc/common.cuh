// Shared device building blocks of the TVC library: element types and
// their in-register decoding, vector loads, and the accumulators.
//
// FP64 on GB300.  The FP64 pipe of this part retires about 1.6 DFMA per SM
// per clock (about 0.5e12 per second), so one DFMA per streamed 8-byte
// element caps an FP64 contraction near 4 TB/s, well under the HBM rate.
// The FP64 accumulators below therefore form most products on the FP32 pipe
// in "float-float" arithmetic: a double a is split by integer operations
// into ah + al (24 + 24 significant bits, exact up to 2^-48 relative), the
// vector entry x into xh + xl (rounded pieces), the leading product ah*xh is
// made error-free with one FMA (Dekker / Kahan TwoProduct), the cross terms
// are added in FP32, and the running sum is kept as an unevaluated pair
// (s, c) updated with Knuth's TwoSum.  Every RB rows the pair is folded into
// an FP64 accumulator.  Elements outside the window where the split is
// exact (|a| outside [2^-64, 2^64), zeros, FP64 subnormals, Inf/NaN, or an x
// entry outside [2^-32, 2^32) that is not zero) take a plain DFMA instead,
// so the result is always an FP64-accurate contraction; only the speed
// depends on the data.  A compile-time share of rows can also be sent to
// the DFMA pipe on purpose, so both pipes work in parallel.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tvc.h"

namespace tvcg {

constexpr int kWarp = 32;

// ------------------------------------------------------------ vector loads

template <int BYTES>
struct RawVec;
template <>
struct RawVec<1> { uint8_t v; };
template <>
struct RawVec<2> { uint16_t v; };
template <>
struct RawVec<4> { uint32_t v; };
template <>
struct RawVec<8> { uint2 v; };
template <>
struct RawVec<16> { uint4 v; };

// Streaming (evict-first) load of BYTES bytes: the tensor is read once.
template <int BYTES>
__device__ __forceinline__ RawVec<BYTES> ld_stream(const void* p) {
  RawVec<BYTES> r;
  if constexpr (BYTES == 16) {
    r.v = __ldcs(reinterpret_cast<const uint4*>(p));
  } else if constexpr (BYTES == 8) {
    r.v = __ldcs(reinterpret_cast<const uint2*>(p));
  } else if constexpr (BYTES == 4) {
    r.v = __ldcs(reinterpret_cast<const unsigned int*>(p));
  } else if constexpr (BYTES == 2) {
    r.v = __ldcs(reinterpret_cast<const unsigned short*>(p));
  } else {
    r.v = __ldcs(reinterpret_cast<const unsigned char*>(p));
  }
  return r;
}

// Plain (generic-address) load: works on shared and global memory.
template <int BYTES>
__device__ __forceinline__ RawVec<BYTES> ld_plain(const void* p) {
  RawVec<BYTES> r;
  if constexpr (BYTES == 16) {
    r.v = *reinterpret_cast<const uint4*>(p);
  } else if constexpr (BYTES == 8) {
    r.v = *reinterpret_cast<const uint2*>(p);
  } else if constexpr (BYTES == 4) {
    r.v = *reinterpret_cast<const unsigned int*>(p);
  } else if constexpr (BYTES == 2) {
    r.v = *reinterpret_cast<const unsigned short*>(p);
  } else {
    r.v = *reinterpret_cast<const unsigned char*>(p);
  }
  return r;
}

template <int BYTES, bool PLAIN>
__device__ __forceinline__ RawVec<BYTES> ld_any(const void* p) {
  if constexpr (PLAIN)
    return ld_plain<BYTES>(p);
  else
    return ld_stream<BYTES>(p);
}

// ------------------------------------------------------ element type traits

// Storage type traits: element type, FP64 or FP32 arithmetic, and decoding
// of VEC consecutive elements into `val` (FP64 for F64, FP32 otherwise).
template <tvc_dtype DT>
struct Elem;

template <>
struct Elem<TVC_F64> {
  using T = double;
  using V = double;  // vector / result type
  using C = double;  // compute type of one element
  static constexpr int kSize = 8;
  template <int VEC, bool PLAIN = false>
  __device__ __forceinline__ static void load(const T* p, C (&val)[VEC]) {
    if constexpr (VEC == 2) {
      RawVec<16> r = ld_any<16, PLAIN>(p);
      val[0] = __hiloint2double((int)r.v.y, (int)r.v.x);
      val[1] = __hiloint2double((int)r.v.w, (int)r.v.z);
    } else {
#pragma unroll
      for (int e = 0; e < VEC; e++) {
        RawVec<8> r = ld_any<8, PLAIN>(p + e);
        val[e] = __hiloint2double((int)r.v.y, (int)r.v.x);
      }
    }
  }
};

template <>
struct Elem<TVC_F32> {
  using T = float;
  using V = float;
  using C = float;
  static constexpr int kSize = 4;
  // Decoding of one 16-byte word of codes (the narrow long-row kernel keeps
  // codes packed until they are used).
  __device__ __forceinline__ static void decode16(const uint4& w, float (&val)[4]) {
    val[0] = __uint_as_float(w.x);
    val[1] = __uint_as_float(w.y);
    val[2] = __uint_as_float(w.z);
    val[3] = __uint_as_float(w.w);
  }
  template <int VEC, bool PLAIN = false>
  __device__ __forceinline__ static void load(const T* p, C (&val)[VEC]) {
    if constexpr (VEC == 4) {
      RawVec<16> r = ld_any<16, PLAIN>(p);
      val[0] = __uint_as_float(r.v.x);
      val[1] = __uint_as_float(r.v.y);
      val[2] = __uint_as_float(r.v.z);
      val[3] = __uint_as_float(r.v.w);
    } else if constexpr (VEC == 2) {
      RawVec<8> r = ld_any<8, PLAIN>(p);
      val[0] = __uint_as_float(r.v.x);
      val[1] = __uint_as_float(r.v.y);
    } else {
#pragma unroll
      for (int e = 0; e < VEC; e++) val[e] = __uint_as_float(ld_any<4, PLAIN>(p + e).v);
    }
  }
};

// FP32 storage with FP64 arithmetic and FP64 vectors (Section 5.5's
// single-double): elements load as binary32 and enter the float-float
// products without the hi/lo split a binary64 element needs.
template <>
struct Elem<TVC_F32D> {
  using T = float;
  using V = double;
  using C = float;
  static constexpr int kSize = 4;
  template <int VEC, bool PLAIN = false>
  __device__ __forceinline__ static void load(const T* p, C (&val)[VEC]) {
    Elem<TVC_F32>::template load<VEC, PLAIN>(p, val);
  }
};

// Storage types whose arithmetic and vectors are FP64.
template <tvc_dtype DT>
inline constexpr bool kF64Acc = (DT == TVC_F64 || DT == TVC_F32D);

// BF16: the code is the upper half of a binary32, so decoding is a shift.
template <>
struct Elem<TVC_BF16> {
  using T = uint16_t;
  using V = float;
  using C = float;
  static constexpr int kSize = 2;
  __device__ __forceinline__ static void decode16(const uint4& w, float (&val)[8]) {
    word2(w.x, val[0], val[1]);
    word2(w.y, val[2], val[3]);
    word2(w.z, val[4], val[5]);
    word2(w.w, val[6], val[7]);
  }
  __device__ __forceinline__ static void word2(uint32_t w, float& lo, float& hi) {
    lo = __uint_as_float(w << 16);
    hi = __uint_as_float(w & 0xFFFF0000u);
  }
  template <int VEC, bool PLAIN = false>
  __device__ __forceinline__ static void load(const T* p, C (&val)[VEC]) {
    if constexpr (VEC == 8) {
      RawVec<16> r = ld_any<16, PLAIN>(p);
      word2(r.v.x, val[0], val[1]);
      word2(r.v.y, val[2], val[3]);
      word2(r.v.z, val[4], val[5]);
      word2(r.v.w, val[6], val[7]);
    } else if constexpr (VEC == 4) {
      RawVec<8> r = ld_any<8, PLAIN>(p);
      word2(r.v.x, val[0], val[1]);
      word2(r.v.y, val[2], val[3]);
    } else if constexpr (VEC == 2) {
      word2(ld_any<4, PLAIN>(p).v, val[0], val[1]);
    } else {
#pragma unroll
      for (int e = 0; e < VEC; e++) val[e] = __uint_as_float(((uint32_t)ld_any<2, PLAIN>(p + e).v) << 16);
    }
  }
};

// FP16 (IEEE binary16): converted two at a time, f16x2 -> two FP32 (exact).
template <>
struct Elem<TVC_F16> {
  using T = uint16_t;
  using V = float;
  using C = float;
  static constexpr int kSize = 2;
  __device__ __forceinline__ static void word2(uint32_t w, float& lo, float& hi) {
    __half2_raw r;
    r.x = (unsigned short)(w & 0xFFFFu);
    r.y = (unsigned short)(w >> 16);
    const float2 f = __half22float2(__half2(r));
    lo = f.x;
    hi = f.y;
  }
  __device__ __forceinline__ static void decode16(const uint4& w, float (&val)[8]) {
    word2(w.x, val[0], val[1]);
    word2(w.y, val[2], val[3]);
    word2(w.z, val[4], val[5]);
    word2(w.w, val[6], val[7]);
  }
  template <int VEC, bool PLAIN = false>
  __device__ __forceinline__ static void load(const T* p, C (&val)[VEC]) {
    if constexpr (VEC == 8) {
      RawVec<16> r = ld_any<16, PLAIN>(p);
      decode16(r.v, val);
    } else if constexpr (VEC == 4) {
      RawVec<8> r = ld_any<8, PLAIN>(p);
      word2(r.v.x, val[0], val[1]);
      word2(r.v.y, val[2], val[3]);
    } else if constexpr (VEC == 2) {
      word2(ld_any<4, PLAIN>(p).v, val[0], val[1]);
    } else {
#pragma unroll
      for (int e = 0; e < VEC; e++) {
        __half_raw h;
        h.x = ld_any<2, PLAIN>(p + e).v;
        val[e] = __half2float(__half(h));
      }
    }
  }
};

// Storage types with per-slab scales (decoded to FP32 in registers).
template <tvc_dtype DT>
inline constexpr bool kNarrow = (DT == TVC_BF16 || DT == TVC_E4M3 || DT == TVC_F16);

// FP8 E4M3 (OCP): decoded two at a time by the hardware e4m3x2 -> f16x2
// conversion, then widened to FP32 (both exact).
template <>
struct Elem<TVC_E4M3> {
  using T = uint8_t;
  using V = float;
  using C = float;
  static constexpr int kSize = 1;
  __device__ __forceinline__ static void decode16(const uint4& w, float (&val)[16]) {
    word4(w.x, val + 0);
    word4(w.y, val + 4);
    word4(w.z, val + 8);
    word4(w.w, val + 12);
  }
  __device__ __forceinline__ static void pair(uint16_t w, float& lo, float& hi) {
    __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)w, __NV_E4M3);
    float2 f = __half22float2(*reinterpret_cast<__half2*>(&h));
    lo = f.x;
    hi = f.y;
  }
  __device__ __forceinline__ static void word4(uint32_t w, float* o) {
    pair((uint16_t)(w & 0xFFFFu), o[0], o[1]);
    pair((uint16_t)(w >> 16), o[2], o[3]);
  }
  template <int VEC, bool PLAIN = false>
  __device__ __forceinline__ static void load(const T* p, C (&val)[VEC]) {
    if constexpr (VEC == 16) {
      RawVec<16> r = ld_any<16, PLAIN>(p);
      word4(r.v.x, val + 0);
      word4(r.v.y, val + 4);
      word4(r.v.z, val + 8);
      word4(r.v.w, val + 12);
    } else if constexpr (VEC == 8) {
      RawVec<8> r = ld_any<8, PLAIN>(p);
      word4(r.v.x, val + 0);
      word4(r.v.y, val + 4);
    } else if constexpr (VEC == 4) {
      word4(ld_any<4, PLAIN>(p).v, val);
    } else {
#pragma unroll
      for (int e = 0; e < VEC; e++) {
        __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)ld_any<1, PLAIN>(p + e).v, __NV_E4M3);
        val[e] = __half2float(*reinterpret_cast<__half*>(&h));
      }
    }
  }
};

// ------------------------------------------------------- float-float parts

// x entry prepared for the emulated FP64 product: x ~= xh + xl (rounded
// pieces).  xh is NaN when x is outside the exact window; such rows use DFMA.
struct XSplit {
  float xh, xl;
};

__device__ __forceinline__ XSplit split_x(double x) {
  XSplit r;
  double ax = fabs(x);
  if (x == 0.0) {
    r.xh = 0.0f;
    r.xl = 0.0f;
  } else if (ax >= 0x1p-32 && ax < 0x1p32) {
    r.xh = __double2float_rn(x);
    r.xl = __double2float_rn(x - (double)r.xh);
  } else {
    r.xh = __int_as_float(0x7FC00000);
    r.xl = 0.0f;
  }
  return r;
}

// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest FP32).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bp = __fsub_rn(s, a);
  float ap = __fsub_rn(s, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// (s, c) += a * x for one FP64 element a (see the file comment).  Lower
// bound of the exact window: exponent field 959 (|a| >= 2^-64), 128 binades.
constexpr uint32_t kDfWindowBase = 959u << 21;

// The out-of-window path is a real call, never an if-converted DFMA that would
// occupy the FP64 pipe for every element; it reads x itself, so the fast path
// needs only the split pieces.
static __device__ __noinline__ double dfma_slow(double a, const double* xp, double d) {
  return fma(a, *xp, d);
}

__device__ __forceinline__ void df_mac(float& s, float& c, double& d, double a, const double* xp,
                                       XSplit xs) {
  const uint32_t lo = (uint32_t)__double2loint(a);
  const uint32_t hi = (uint32_t)__double2hiint(a);
  const uint32_t win = hi * 2u - kDfWindowBase;
  if (win < (1u << 28) && xs.xh == xs.xh) {
    // ah: rebias the exponent (1023 -> 127) and keep the top 23 fraction bits.
    const uint32_t hb = __funnelshift_l(lo, hi - 0x38000000u, 3) | (hi & 0x80000000u);
    const float ah = __uint_as_float(hb);
    // al: the remaining 29 fraction bits times 2^(e-1075), signed like a.
    const float sc = __uint_as_float((hb & 0xFF800000u) - 0x1A000000u);
    const float al = __fmul_rn(__uint2float_rn(lo & 0x1FFFFFFFu), sc);
    const float p = __fmul_rn(ah, xs.xh);
    float e = __fmaf_rn(ah, xs.xh, -p);
    e = __fmaf_rn(ah, xs.xl, e);
    e = __fmaf_rn(al, xs.xh, e);
    float t, err;
    two_sum(s, p, t, err);
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
  } else {
    d = dfma_slow(a, xp, d);
  }
}

// (s, c) += a * x for one binary32 element a (FP32 storage, FP64
// arithmetic): a is exact as it stands, so only the TwoProduct against the
// two pieces of x remains.  Window: |a| in [2^-64, 2^64) (biased exponent
// 63 .. 190), zeros, subnormals and Inf/NaN take the exact DFMA.
static __device__ __noinline__ double dfma_slow_f(float a, const double* xp, double d) {
  return fma((double)a, *xp, d);
}

// Nonzero when the binary32 a is outside its window: with the sign shifted
// out, exponent field - 63 wraps below the window, and 128 binades span
// exactly 2^31, so bit 31 of the difference is the test.
__device__ __forceinline__ uint32_t df_out_of_window(float a) {
  return (((uint32_t)__float_as_uint(a) << 1) - (63u << 24)) >> 31;
}

__device__ __forceinline__ void df_mac_fast(float& s, float& c, float a, XSplit xs) {
  const float p = __fmul_rn(a, xs.xh);
  float e = __fmaf_rn(a, xs.xh, -p);
  e = __fmaf_rn(a, xs.xl, e);
  float t, err;
  two_sum(s, p, t, err);
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

__device__ __forceinline__ void df_mac(float& s, float& c, double& d, float a, const double* xp, XSplit xs) {
  if (df_out_of_window(a) == 0 && xs.xh == xs.xh) {
    df_mac_fast(s, c, a, xs);
  } else {
    d = dfma_slow_f(a, xp, d);
  }
}

// df_mac without the window test, for elements already known to be in the
// window (see df_out_of_window); x must be in its window too.
__device__ __forceinline__ void df_mac_fast(float& s, float& c, double a, XSplit xs) {
  const uint32_t lo = (uint32_t)__double2loint(a);
  const uint32_t hi = (uint32_t)__double2hiint(a);
  const uint32_t hb = __funnelshift_l(lo, hi - 0x38000000u, 3) | (hi & 0x80000000u);
  const float ah = __uint_as_float(hb);
  const float sc = __uint_as_float((hb & 0xFF800000u) - 0x1A000000u);
  const float al = __fmul_rn(__uint2float_rn(lo & 0x1FFFFFFFu), sc);
  const float p = __fmul_rn(ah, xs.xh);
  float e = __fmaf_rn(ah, xs.xh, -p);
  e = __fmaf_rn(ah, xs.xl, e);
  e = __fmaf_rn(al, xs.xh, e);
  float t, err;
  two_sum(s, p, t, err);
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

// The float-float split a = ah + al of an in-window double (the split of
// df_mac_fast on its own, for kernels that reuse one element's pieces
// against several x).
__device__ __forceinline__ void df_split(double a, float& ah, float& al) {
  const uint32_t lo = (uint32_t)__double2loint(a);
  const uint32_t hi = (uint32_t)__double2hiint(a);
  const uint32_t hb = __funnelshift_l(lo, hi - 0x38000000u, 3) | (hi & 0x80000000u);
  ah = __uint_as_float(hb);
  const float sc = __uint_as_float((hb & 0xFF800000u) - 0x1A000000u);
  al = __fmul_rn(__uint2float_rn(lo & 0x1FFFFFFFu), sc);
}

// df_mac_fast with the window bit of a ORed into `bad`: kernels run every
// element through it and redo the (rare) results that met an element
// outside the window with DFMA.  An x outside its window needs no test: its
// NaN pieces make the pair NaN.
__device__ __forceinline__ void df_step(float& s, float& c, uint32_t& bad, double a, XSplit xs);

// Nonzero when a is outside the exact window of the float-float split
// (two integer operations; OR it over many elements, test once).
__device__ __forceinline__ uint32_t df_out_of_window(double a) {
  return ((uint32_t)__double2hiint(a) * 2u - kDfWindowBase) >> 28;
}

__device__ __forceinline__ void df_step(float& s, float& c, uint32_t& bad, double a, XSplit xs) {
  bad |= df_out_of_window(a);
  df_mac_fast(s, c, a, xs);
}

__device__ __forceinline__ void df_step(float& s, float& c, uint32_t& bad, float a, XSplit xs) {
  bad |= df_out_of_window(a);
  df_mac_fast(s, c, a, xs);
}

// Adds an FP64 partial d into the float-float pair (s, c): d is split like
// an element (ah + al, integer operations only) when it lies in the window
// (the callers keep out-of-window partials in FP64); zero is skipped.
__device__ __forceinline__ void df_add_double(float& s, float& c, double d) {
  float hi, lo;
  if (df_out_of_window(d) == 0) {
    const uint32_t l = (uint32_t)__double2loint(d);
    const uint32_t h = (uint32_t)__double2hiint(d);
    const uint32_t hb = __funnelshift_l(l, h - 0x38000000u, 3) | (h & 0x80000000u);
    hi = __uint_as_float(hb);
    lo = __fmul_rn(__uint2float_rn(l & 0x1FFFFFFFu), __uint_as_float((hb & 0xFF800000u) - 0x1A000000u));
  } else if (d == 0.0) {
    return;
  } else {
    hi = __double2float_rn(d);
    lo = __double2float_rn(d - (double)hi);
  }
  float t, err;
  two_sum(s, hi, t, err);
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, lo));
}

// ------------------------------------------------------------ accumulators

// FP64 accumulator for VEC columns: float-float pairs plus an FP64 total.
template <int VEC>
struct AccF64 {
  float s[VEC], c[VEC];
  double d[VEC];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int e = 0; e < VEC; e++) {
      s[e] = 0.0f;
      c[e] = 0.0f;
      d[e] = 0.0;
    }
  }
  template <class A>  // double (FP64 storage) or float (FP32 storage)
  __device__ __forceinline__ void emul(const A (&a)[VEC], const double* xp, XSplit xs) {
#pragma unroll
    for (int e = 0; e < VEC; e++) df_mac(s[e], c[e], d[e], a[e], xp, xs);
  }
  // One column, its own x entry (row-wise kernels).
  template <class A>
  __device__ __forceinline__ void emul1(int e, A a, const double* xp, XSplit xs) {
    df_mac(s[e], c[e], d[e], a, xp, xs);
  }
  template <class A>
  __device__ __forceinline__ void dfma(const A (&a)[VEC], double x) {
#pragma unroll
    for (int e = 0; e < VEC; e++) d[e] = fma((double)a[e], x, d[e]);
  }
  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int e = 0; e < VEC; e++) {
      d[e] += (double)s[e];
      d[e] += (double)c[e];
      s[e] = 0.0f;
      c[e] = 0.0f;
    }
  }
  __device__ __forceinline__ double result(int e) const { return d[e]; }
};

// FP32 accumulator for VEC columns: plain FMAs within a block of rows, the
// block sums folded into a compensated pair (S, C) with TwoSum.
template <int VEC>
struct AccF32 {
  float a[VEC], S[VEC], C[VEC];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int e = 0; e < VEC; e++) {
      a[e] = 0.0f;
      S[e] = 0.0f;
      C[e] = 0.0f;
    }
  }
  __device__ __forceinline__ void mac(const float (&v)[VEC], float x) {
#pragma unroll
    for (int e = 0; e < VEC; e++) a[e] = __fmaf_rn(v[e], x, a[e]);
  }
  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int e = 0; e < VEC; e++) {
      float t, err;
      two_sum(S[e], a[e], t, err);
      S[e] = t;
      C[e] = __fadd_rn(C[e], err);
      a[e] = 0.0f;
    }
  }
  __device__ __forceinline__ float result(int e) const { return __fadd_rn(S[e], C[e]); }
};

// Compensated FP32 sum helper for reductions of partial results.
struct KahanF32 {
  float S = 0.0f, C = 0.0f;
  __device__ __forceinline__ void add(float v) {
    float t, err;
    two_sum(S, v, t, err);
    S = t;
    C = __fadd_rn(C, err);
  }
  __device__ __forceinline__ float value() const { return __fadd_rn(S, C); }
};

}  // namespace tvcg
