// Batched contractions, adjoints and power methods over many independent
// FP32 tensors of uneven order and shape, each batch in one persistent
// launch (the GPU counterpart of the paper's task-based execution, Section
// 4.3, where many TVCs overlap instead of joining after each one).
//
// Contraction and adjoints: the host cuts every tensor (largest first) into
// work items of about 2^20 elements (output ranges of the forward
// contraction, slab x row rectangles of gx and gA) and uploads the
// descriptors and items into the workspace; a persistent kernel of a few
// blocks per SM pulls items from an atomic work counter.  gx items of one
// tensor leave partial sums that the tensor's last item adds in a fixed
// order.  Power methods: one block runs every sweep of one tensor.  With
// TVC_BATCH_PREUPLOADED the descriptors of a previous call are reused and a
// call issues only a memset and one kernel, so it can be captured in a CUDA
// graph and replayed.
//
// Forward contraction of rows v == 1: a group of G lanes (G a power of two
// <= 32) computes one output, its lanes splitting the row; the autotuner
// picks G per shape class (n_k rounded to a power of two) by timing the
// candidates, untuned classes use a fixed rule.  For v >= 2 one thread
// computes one output, coalesced along l.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace tvcg {
namespace {

constexpr int kBBT = 256;        // threads per block
constexpr int kBBlocksPerSM = 6;

struct BItem {
  const float* A;
  const float* x;
  float* y;
  const float* gy;
  float* gx;
  float* gA;
  int64_t u, nk, v;
  int gf;         // lanes per output of the forward contraction
  int gxk;        // gx items (slab ranges) of this tensor
  int64_t gxp;    // their partials: floats [gxp, gxp + gxk * nk) of the partial area (gxk > 1)
};

struct HItem {
  const float* A;
  int d;
  int gsel[TVC_MAX_ORDER];
  int64_t dims[TVC_MAX_ORDER];
  float* x[TVC_MAX_ORDER];
  double* lam;
  int* status;
};

// ---------------------------------------------------- block-level routines

// y[o] = sum_j A[(i*nk + j)*v + l] x[j], o = i*v + l < u*v; G lanes per output.
__device__ void blk_tvc(const float* __restrict__ A, int64_t u, int64_t nk, int64_t v, const float* __restrict__ x,
                        float* __restrict__ y, int G, int64_t o_begin = 0, int64_t o_end = -1) {
  const int64_t uv = (o_end < 0) ? u * v : o_end;
  if (v >= 2) {
    // One thread per output o = (i, l): the pair is found by one division
    // and then advanced by the block stride; sixteen rows of n_k in flight
    // through pointer increments (one block streams at the rate its bytes in
    // flight allow), only the last (< 8) rows predicated.
    int64_t o = o_begin + threadIdx.x;
    if (o >= uv) return;
    int64_t i = o / v, l = o - i * v;
    const int64_t stride = kBBT;
    const int64_t di = stride / v, dl = stride - di * v;
    for (; o < uv; o += stride) {
      const float* p = A + i * nk * v + l;
      float acc0 = 0.0f, acc1 = 0.0f;
      int64_t jj = 0;
      for (; jj + 16 <= nk; jj += 16, p += 16 * v) {  // 16 rows in flight (64 B per thread)
        float av[16];
#pragma unroll
        for (int q = 0; q < 16; q++) av[q] = __ldcs(p + q * v);
#pragma unroll
        for (int q = 0; q < 16; q += 2) {
          acc0 = __fmaf_rn(av[q], __ldg(x + jj + q), acc0);
          acc1 = __fmaf_rn(av[q + 1], __ldg(x + jj + q + 1), acc1);
        }
      }
      if (jj + 8 <= nk) {
        float av[8];
#pragma unroll
        for (int q = 0; q < 8; q++) av[q] = __ldcs(p + q * v);
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
          acc0 = __fmaf_rn(av[q], __ldg(x + jj + q), acc0);
          acc1 = __fmaf_rn(av[q + 1], __ldg(x + jj + q + 1), acc1);
        }
        jj += 8;
        p += 8 * v;
      }
      if (jj < nk) {
        float av[7];
#pragma unroll
        for (int q = 0; q < 7; q++) av[q] = (jj + q < nk) ? __ldcs(p + q * v) : 0.0f;
#pragma unroll
        for (int q = 0; q < 7; q++)
          if (jj + q < nk) acc0 = __fmaf_rn(av[q], __ldg(x + jj + q), acc0);
      }
      y[o] = acc0 + acc1;
      i += di;
      l += dl;
      if (l >= v) {
        l -= v;
        i++;
      }
    }
    return;
  }
  // v == 1 (rows): a group of G lanes per row, eight predicated loads in
  // flight per lane (short rows too), shuffle reduction.
  const int lane = threadIdx.x & 31;
  const int p = lane & (G - 1);
  const int gw = 32 / G;  // groups per warp
  const int64_t ngroups = (int64_t)(kBBT / 32) * gw;
  for (int64_t base = o_begin + (int64_t)(threadIdx.x >> 5) * gw; base < uv; base += ngroups) {
    const int64_t o = base + lane / G;
    float acc = 0.0f;
    if (o < uv) {
      const float* row = A + o * nk;
      for (int64_t j = p; j < nk; j += 8 * G) {
        float av[8], xv[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const bool ok = j + q * G < nk;
          av[q] = ok ? __ldcs(row + j + q * G) : 0.0f;
          xv[q] = ok ? __ldg(x + j + q * G) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 8; q++) acc = __fmaf_rn(av[q], xv[q], acc);
      }
    }
    for (int off = G / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
    if (o < uv && p == 0) y[o] = acc;
  }
}

// The power method's two passes over A (v >= 2): where v is even and A is
// 8-byte aligned each thread takes two adjacent outputs and loads pairs,
// twice the bytes in flight per thread for the same sixteen rows (a block
// of the register-held contraction streams at the rate its bytes in flight
// allow); otherwise blk_tvc.
__device__ void blk_tvc_pass(const float* __restrict__ A, int64_t u, int64_t nk, int64_t v,
                             const float* __restrict__ x, float* __restrict__ y, int G) {
  if (v % 2 != 0 || (reinterpret_cast<uintptr_t>(A) & 7) != 0) {
    blk_tvc(A, u, nk, v, x, y, G);
    return;
  }
  const int64_t uv2 = u * v / 2;  // output pairs
  int64_t q2 = threadIdx.x;
  if (q2 >= uv2) return;
  const int64_t v2 = v / 2;
  int64_t i = q2 / v2, l = 2 * (q2 - i * v2);
  const int64_t di = kBBT / v2, dl = 2 * (kBBT - di * v2);
  for (; q2 < uv2; q2 += kBBT) {
    const float* p = A + i * nk * v + l;
    float a0 = 0.0f, a1 = 0.0f;
    int64_t jj = 0;
    for (; jj + 16 <= nk; jj += 16, p += 16 * v) {
      float2 av[16];
#pragma unroll
      for (int q = 0; q < 16; q++) av[q] = __ldcs(reinterpret_cast<const float2*>(p + q * v));
#pragma unroll
      for (int q = 0; q < 16; q++) {
        const float xv = __ldg(x + jj + q);
        a0 = __fmaf_rn(av[q].x, xv, a0);
        a1 = __fmaf_rn(av[q].y, xv, a1);
      }
    }
    for (; jj < nk; jj++, p += v) {
      const float2 av = __ldcs(reinterpret_cast<const float2*>(p));
      const float xv = __ldg(x + jj);
      a0 = __fmaf_rn(av.x, xv, a0);
      a1 = __fmaf_rn(av.y, xv, a1);
    }
    y[i * v + l] = a0;
    y[i * v + l + 1] = a1;
    i += di;
    l += dl;
    if (l >= v) {
      l -= v;
      i++;
    }
  }
}

// gA[(i*nk + j)*v + l] = gy[i*v + l] * x[j] over slabs i in [i0, i1) and
// rows j in [j0, j1), with coalesced stores: threads own columns l (v >= 32)
// or positions q = j*v + l of the slab (v < 32, whole slabs).
__device__ void blk_gA(const float* __restrict__ gy, const float* __restrict__ x, float* __restrict__ gA, int64_t nk,
                       int64_t v, int64_t i0, int64_t i1, int64_t j0, int64_t j1) {
  if (v >= 32) {
    for (int64_t l = threadIdx.x; l < v; l += kBBT)
      for (int64_t i = i0; i < i1; i++) {
        const float g = __ldg(gy + i * v + l);
        float* p = gA + (i * nk + j0) * v + l;
        for (int64_t j = j0; j < j1; j++, p += v) __stcs(p, g * __ldg(x + j));
      }
  } else {
    const int64_t S = nk * v;
    for (int64_t q = threadIdx.x; q < S; q += kBBT) {
      const int64_t j = q / v, l = q - j * v;
      const float xj = __ldg(x + j);
      for (int64_t i = i0; i < i1; i++) __stcs(gA + i * S + q, __ldg(gy + i * v + l) * xj);
    }
  }
}

// w[c] = prod_{m < nm} x_m[digit_m(c)]
__device__ void blk_outer(float* w, int nm, const int64_t* dims, float* const* xs) {
  int64_t len = 1;
  for (int m = 0; m < nm; m++) len *= dims[m];
  for (int64_t c = threadIdx.x; c < len; c += kBBT) {
    int64_t rem = c;
    float acc = 1.0f;
    int64_t dig[TVC_MAX_ORDER];
    for (int m = nm - 1; m >= 0; m--) {
      dig[m] = rem % dims[m];
      rem /= dims[m];
    }
    acc = xs[0][dig[0]];
    for (int m = 1; m < nm; m++) acc *= xs[m][dig[m]];
    w[c] = acc;
  }
}

// x = z / ||z|| with the norm in FP64; returns the norm (all threads).
__device__ double blk_normalize(const float* z, float* x, int64_t n, double* red) {
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kBBT) s = fma((double)z[i], (double)z[i], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = kBBT / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  const double sigma = sqrt(red[0]);
  __syncthreads();
  if (isfinite(sigma) && sigma > 0.0)
    for (int64_t i = threadIdx.x; i < n; i += kBBT) x[i] = (float)((double)z[i] / sigma);
  __syncthreads();
  return sigma;
}

__device__ int grab(int* counter, int* slot) {
  __syncthreads();
  if (threadIdx.x == 0) *slot = atomicAdd(counter, 1);
  __syncthreads();
  return *slot;
}

// ------------------------------------------------------------ the kernels

// A unit of work: kind 0 = outputs [a0, a1) of the forward contraction,
// 1 = gx over slabs [a0, a1) and rows j in [c0, c1) (slab range e0 of the
// tensor's gxk, e1 gx items in all), 2 = gA over slabs [a0, a1) and rows
// [c0, c1).
struct WItem {
  int b, kind;
  int64_t a0, a1, c0, c1;
  int e0, e1;
};

// gx over a rectangle of one tensor: slabs [i0, i1) x rows j in [j0, j1)
// (item ks of the tensor's gxk slab ranges):
//   part[j] = sum_{i in [i0,i1), l < v} A[(i*nk + j)*v + l] gy[i*v + l].
// Rows of v >= 32 go to warps: warp w takes the slabs i = i0 + w (mod 8) of
// every j (or, when the item has fewer than 8 slabs, the w-th 32-aligned
// segment of every row), lanes stride over l; each warp's sum for j (FP32
// folded every 64 products into a compensated pair, then a fixed xor tree) goes
// to red[w][j - j0] and the 8 warp sums are added in w order (j1 - j0 <=
// kGxJ).  Rows of v < 32 go to columns: the item's columns c = j*v + l
// (contiguous in every slab) are taken in chunks of at most kBBT; a chunk
// narrower than the block gives the spare threads alternate slabs (phases).
// Each thread streams its column down its slabs (eight in flight, folded
// every 64 slabs), the phases of a column are added in phase order and the
// columns of a j in l order.  With gxk > 1 the slab ranges write partials
// [ks][j] and the tensor's last item to finish (counted per tensor) sums them
// in slab-range order into gx and resets the counter: deterministic, no
// waiting.
constexpr int64_t kGxWarpRows = 32;  // v at or above which rows go to warps
constexpr int64_t kGxJ = 256;        // rows j per warp-mapped item

__device__ void blk_gx_rect(const BItem& it, int64_t i0, int64_t i1, int64_t j0, int64_t j1, int ks, int items,
                            int* cnt, float* partials, float* red, int* flag) {
  const int64_t S = it.nk * it.v, v = it.v;
  float* dst = (it.gxk > 1) ? partials + it.gxp + (int64_t)ks * it.nk : it.gx;
  const int t = threadIdx.x;
  if (v >= kGxWarpRows) {
    const int w = t >> 5, lane = t & 31;
    const bool phase = i1 - i0 >= 8;
    const int64_t seg = phase ? v : ((v + 8 * 32 - 1) / (8 * 32)) * 32;
    const int64_t ls = phase ? 0 : min((int64_t)w * seg, v);
    const int64_t L = min(seg, v - ls);
    const int64_t ib = phase ? i0 + w : i0, di = phase ? 8 : 1;
    for (int64_t j = j0; j < j1; j++) {
      KahanF32 tot;
      int64_t i = ib;
      const float* a = it.A + (i * it.nk + j) * v + ls;
      const float* g = it.gy + i * v + ls;
      // folded every 16 lane passes (at most 64 products per partial sum)
      for (; i + 3 * di < i1; i += 4 * di, a += 4 * di * S, g += 4 * di * v)
        for (int64_t lb = 0; lb < L; lb += 16 * 32) {
          const int64_t le = min(lb + 16 * 32, L);
          float acc = 0.0f;
          for (int64_t l = lb + lane; l < le; l += 32) {
            const float x0 = __ldcs(a + l), x1 = __ldcs(a + di * S + l);
            const float x2 = __ldcs(a + 2 * di * S + l), x3 = __ldcs(a + 3 * di * S + l);
            const float y0 = __ldg(g + l), y1 = __ldg(g + di * v + l);
            const float y2 = __ldg(g + 2 * di * v + l), y3 = __ldg(g + 3 * di * v + l);
            acc = __fmaf_rn(x0, y0, acc);
            acc = __fmaf_rn(x1, y1, acc);
            acc = __fmaf_rn(x2, y2, acc);
            acc = __fmaf_rn(x3, y3, acc);
          }
          tot.add(acc);
        }
      for (; i < i1; i += di, a += di * S, g += di * v)
        for (int64_t lb = 0; lb < L; lb += 64 * 32) {
          const int64_t le = min(lb + 64 * 32, L);
          float acc = 0.0f;
          for (int64_t l = lb + lane; l < le; l += 32) acc = __fmaf_rn(__ldcs(a + l), __ldg(g + l), acc);
          tot.add(acc);
        }
      float sw = tot.value();
      for (int off = 16; off > 0; off >>= 1) sw = __fadd_rn(sw, __shfl_xor_sync(0xffffffffu, sw, off));
      if (lane == 0) red[w * kGxJ + (j - j0)] = sw;
    }
    __syncthreads();
    for (int64_t j = j0 + t; j < j1; j += kBBT) {
      float sj = red[j - j0];
      for (int q = 1; q < kBBT / 32; q++) sj = __fadd_rn(sj, red[q * kGxJ + (j - j0)]);
      dst[j] = sj;
    }
    __syncthreads();
  } else {
    const int64_t C = (j1 - j0) * v;  // the item's columns in one slab
    const int CW = (int)min(C, (int64_t)kBBT);
    const int P = kBBT / CW;  // slab phases
    const int ph = t / CW, cc = t - (t / CW) * CW;
    for (int64_t cb = 0; cb < C; cb += CW) {
      const int64_t c = j0 * v + cb + cc;  // column within the slab
      float acc = 0.0f;
      KahanF32 tot;
      if (ph < P && cb + cc < C) {
        const int64_t l = c - (c / v) * v;
        const int64_t di = P;
        const float* a = it.A + (i0 + ph) * S + c;
        const float* g = it.gy + (i0 + ph) * v + l;
        int64_t i = i0 + ph;
        int blk = 0;
        for (; i + 7 * di < i1; i += 8 * di, a += 8 * di * S, g += 8 * di * v) {
          float av[8], gv[8];
#pragma unroll
          for (int q = 0; q < 8; q++) {
            av[q] = __ldcs(a + q * di * S);
            gv[q] = __ldg(g + q * di * v);
          }
#pragma unroll
          for (int q = 0; q < 8; q++) acc = __fmaf_rn(av[q], gv[q], acc);
          if (++blk == 8) {
            tot.add(acc);
            acc = 0.0f;
            blk = 0;
          }
        }
        for (; i < i1; i += di, a += di * S, g += di * v) acc = __fmaf_rn(__ldcs(a), __ldg(g), acc);
        tot.add(acc);
      }
      red[t] = (ph < P && cb + cc < C) ? tot.value() : 0.0f;
      __syncthreads();
      if (t < CW && P > 1) {  // the phases of column cc, in phase order
        float sc = red[t];
        for (int q = 1; q < P; q++) sc = __fadd_rn(sc, red[q * CW + t]);
        red[t] = sc;
      }
      __syncthreads();
      // per j of the chunk: its columns in l order, added in chunk order
      const int64_t c0 = j0 * v + cb, c1 = min(c0 + CW, j1 * v);
      for (int64_t j = c0 / v + t; j * v < c1; j += kBBT) {
        const int64_t a0 = max(j * v, c0), a1 = min((j + 1) * v, c1);
        float sj = 0.0f;
        for (int64_t q = a0; q < a1; q++) sj = __fadd_rn(sj, red[q - c0]);
        dst[j] = (a0 == j * v) ? sj : __fadd_rn(dst[j], sj);  // the chunk holding l = 0 starts j
      }
      __syncthreads();
    }
  }
  if (it.gxk > 1) {
    __threadfence();
    __syncthreads();
    if (t == 0) *flag = (atomicAdd(cnt, 1) == items - 1);
    __syncthreads();
    if (*flag) {
      __threadfence();
      const float* Pp = partials + it.gxp;
      for (int64_t j = t; j < it.nk; j += kBBT) {
        KahanF32 sum;
        for (int q = 0; q < it.gxk; q++) sum.add(__ldcg(Pp + (int64_t)q * it.nk + j));
        it.gx[j] = sum.value();
      }
      if (t == 0) *cnt = 0;  // ready for the next launch
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kBBT, 6) tvc_batched_kernel(const BItem* __restrict__ items,
                                                           const WItem* __restrict__ work, int nwork, int* counter,
                                                           int* gx_counters, float* gx_partials) {
  __shared__ int slot;
  __shared__ float red[(kBBT / 32) * kGxJ];
  __shared__ int last_flag;
  for (int w = grab(counter, &slot); w < nwork; w = grab(counter, &slot)) {
    const WItem wi = work[w];
    const BItem it = items[wi.b];
    if (wi.kind == 0)
      blk_tvc(it.A, it.u, it.nk, it.v, it.x, it.y, it.gf, wi.a0, wi.a1);
    else if (wi.kind == 1)
      blk_gx_rect(it, wi.a0, wi.a1, wi.c0, wi.c1, wi.e0, wi.e1, gx_counters + wi.b, gx_partials, red, &last_flag);
    else
      blk_gA(it.gy, it.x, it.gA, it.nk, it.v, wi.a0, wi.a1, wi.c0, wi.c1);
  }
}

// One block runs every sweep of one tensor's power method (the schedule of
// the single-tensor path: T = A x_1 x_1, W_1 = A x_0 x_0, W_j = W_{j-1} x_{j-1} ...,
// the trailing contractions against the outer product of the trailing
// vectors).  scratch: per block, 3 buffers of `slen` floats plus z.
__global__ void __launch_bounds__(kBBT) hopm_batched_kernel(const HItem* __restrict__ items, int count, int iters,
                                                            int* counter, float* scratch, int64_t slen, int64_t zlen) {
  __shared__ int slot;
  __shared__ double red[kBBT];
  float* S1 = scratch + (int64_t)blockIdx.x * (3 * slen + zlen);
  float* S2 = S1 + slen;
  float* Wv = S2 + slen;
  float* z = Wv + slen;
  for (int b = grab(counter, &slot); b < count; b = grab(counter, &slot)) {
    const HItem& it = items[b];
    const int d = it.d;
    const int64_t* n = it.dims;
    int64_t N = 1;
    for (int m = 0; m < d; m++) N *= n[m];
    int status = TVC_OK;
    double sigma = 0.0;
    for (int t = 0; t < iters && status == TVC_OK; t++) {
      float* prev = S1;
      float* next = S2;
      for (int j = 0; j < d && status == TVC_OK; j++) {
        const float* zz = z;
        if (d == 2) {
          // z_j = A x_{1-j} x_{1-j}
          if (j == 0)
            blk_tvc(it.A, n[0], n[1], 1, it.x[1], z, it.gsel[1]);
          else
            blk_tvc(it.A, 1, n[0], n[1], it.x[0], z, it.gsel[0]);
        } else if (j < 2) {
          int64_t rest2 = 1;
          for (int m = 2; m < d; m++) rest2 *= n[m];
          if (j == 0)
            blk_tvc_pass(it.A, n[0], n[1], rest2, it.x[1], S1, it.gsel[1]);  // T = A x_1 x_1
          else
            blk_tvc_pass(it.A, 1, n[0], N / n[0], it.x[0], S1, it.gsel[0]);  // W_1 = A x_0 x_0
          __syncthreads();
          const float* wvec = it.x[2];
          if (d > 3) {
            blk_outer(Wv, d - 2, n + 2, it.x + 2);
            __syncthreads();
            wvec = Wv;
          }
          blk_tvc(S1, n[j], rest2, 1, wvec, z, 32);
          prev = S1;
          next = S2;
        } else {
          int64_t rest = 1;
          for (int m = j; m < d; m++) rest *= n[m];
          blk_tvc(prev, 1, n[j - 1], rest, it.x[j - 1], next, 1);  // W_j = W_{j-1} x_{j-1}
          __syncthreads();
          if (j == d - 1) {
            zz = next;
          } else {
            const float* wvec = it.x[d - 1];
            if (j < d - 2) {
              blk_outer(Wv, d - j - 1, n + j + 1, it.x + j + 1);
              __syncthreads();
              wvec = Wv;
            }
            blk_tvc(next, n[j], rest / n[j], 1, wvec, z, 32);
          }
          float* tmp = prev;
          prev = next;
          next = tmp;
        }
        __syncthreads();
        sigma = blk_normalize(zz, it.x[j], n[j], red);
        if (!isfinite(sigma)) status = TVC_ERR_NONFINITE;
        else if (sigma == 0.0) status = TVC_ERR_ZERO_NORM;
      }
    }
    if (threadIdx.x == 0) {
      if (it.lam) *it.lam = sigma;
      if (it.status) *it.status = status;
    }
  }
}

// ------------------------------------------------------------------ host --

int64_t clog2(int64_t x) {
  int64_t r = 0;
  while ((int64_t(1) << r) < x) r++;
  return r;
}

// Autotuner cache of the forward contraction: (log2 v, log2 n_k) -> G.
std::mutex g_tune_mu;
std::map<std::pair<int, int>, int> g_tune;
std::map<void*, int> g_nwork;  // work items uploaded per workspace

int rule_G(int64_t nk, int64_t v) {  // lanes splitting n_k per forward output
  if (v >= 32) return 1;
  if (v >= 8) return 4;
  return nk >= 64 ? 32 : 8;
}

int pick_G(int64_t nk, int64_t v) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find({(int)clog2(v), (int)clog2(nk)});
  return it != g_tune.end() ? it->second : rule_G(nk, v);
}

struct BLayout {
  size_t off_counter = 0, off_items = 0, off_scratch = 0, off_gxcnt = 0, off_gxpart = 0, total = 0;
  int64_t slen = 0, zlen = 0;
  int blocks = 0;
};

// Work of about this many elements per item (a few MB): large tensors
// spread over many blocks, small ones make a single item.
constexpr int64_t kItemElems = 1 << 20;

int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

int64_t assign_gx(std::vector<BItem>* items);

// Rectangle of a gx item: jr rows j by sr slabs, about kItemElems elements.
// Warp-mapped rows (v >= 32) take every slab of a j before cutting the slabs
// and keep 8 slabs (one per warp) where the tensor has them; column-mapped
// rows take whole slab widths.
void gx_rect(const BItem& it, int64_t* jr, int64_t* sr) {
  const int64_t v = std::max<int64_t>(1, it.v);
  if (v >= kGxWarpRows)  // whole slab ranges per j first; at most kGxJ rows, 8 slabs when there are
    *jr = std::max<int64_t>(1, std::min<int64_t>(std::min(it.nk, kGxJ), kItemElems / std::max<int64_t>(1, it.u * v)));
  else  // whole slab widths first (coalesced columns)
    *jr = std::max<int64_t>(1, std::min<int64_t>(it.nk, kItemElems / v));
  *sr = std::max<int64_t>(1, std::min<int64_t>(it.u, kItemElems / (*jr * v)));
  if (v >= kGxWarpRows) *sr = std::max(*sr, std::min<int64_t>(it.u, 8));
}

void make_work(std::vector<BItem>& items, std::vector<WItem>* work) {
  assign_gx(&items);
  work->clear();
  for (int b = 0; b < (int)items.size(); b++) {
    const BItem& it = items[b];
    const int64_t uv = it.u * it.v;
    if (it.y) {
      const int64_t per = std::max<int64_t>(256, cdiv64(kItemElems, it.nk) / 256 * 256);
      for (int64_t o = 0; o < uv; o += per) work->push_back({b, 0, o, std::min(uv, o + per), 0, 0, 0, 0});
    }
    if (it.gx) {  // rectangles (see assign_gx), partials summed by the tensor's last item
      int64_t jr, sr;
      gx_rect(it, &jr, &sr);
      const int nitems = (int)(cdiv64(it.u, sr) * cdiv64(it.nk, jr));
      int ks = 0;
      for (int64_t i = 0; i < it.u; i += sr, ks++)
        for (int64_t j = 0; j < it.nk; j += jr)
          work->push_back({b, 1, i, std::min(it.u, i + sr), j, std::min(it.nk, j + jr), ks, nitems});
    }
    if (it.gA) {
      const int64_t S = it.nk * it.v;
      if (it.v >= 32) {
        // rectangles of slabs x rows
        const int64_t rows = std::max<int64_t>(1, std::min<int64_t>(it.nk, kItemElems / it.v));
        const int64_t slabs = std::max<int64_t>(1, kItemElems / (rows * it.v));
        for (int64_t i = 0; i < it.u; i += slabs)
          for (int64_t j = 0; j < it.nk; j += rows)
            work->push_back({b, 2, i, std::min(it.u, i + slabs), j, std::min(it.nk, j + rows), 0, 0});
      } else {
        const int64_t slabs = std::max<int64_t>(1, kItemElems / S);
        for (int64_t i = 0; i < it.u; i += slabs)
          work->push_back({b, 2, i, std::min(it.u, i + slabs), 0, it.nk, 0, 0});
      }
    }
  }
}

// Workspace of a tensor batch: header, descriptors, work items (the exact
// count, from the same construction the call uses).
tvc_status check_tvc_descs(const tvc_batch_desc* d, int count, std::vector<BItem>* items);

// gx items per tensor (slab ranges of about kItemElems elements) and the
// offsets of their partials; called on every item list before make_work.
int64_t assign_gx(std::vector<BItem>* items) {
  int64_t off = 0;
  for (BItem& it : *items) {
    it.gxk = 0;
    it.gxp = 0;
    if (!it.gx) continue;
    int64_t jr, sr;
    gx_rect(it, &jr, &sr);
    it.gxk = (int)cdiv64(it.u, sr);
    if (it.gxk > 1) {
      it.gxp = off;
      off += (int64_t)it.gxk * it.nk;
    }
  }
  return off;
}

BLayout layout_tvc_items(const std::vector<BItem>& items, size_t nwork) {
  BLayout L;
  L.off_counter = 0;
  L.off_items = 256;
  L.off_scratch = L.off_items + align_up(items.size() * sizeof(BItem), 256);
  L.off_gxcnt = L.off_scratch + align_up(nwork * sizeof(WItem), 256);
  int64_t nparts = 0;
  for (const BItem& it : items)
    if (it.gxk > 1) nparts = std::max<int64_t>(nparts, it.gxp + (int64_t)it.gxk * it.nk);
  L.off_gxpart = L.off_gxcnt + align_up(items.size() * sizeof(int), 256);
  L.total = L.off_gxpart + align_up((size_t)std::max<int64_t>(1, nparts) * sizeof(float), 256);
  L.blocks = device_sms() * kBBlocksPerSM;
  return L;
}

BLayout layout_hopm(const hopm_batch_desc* d, int count) {
  BLayout L;
  L.blocks = device_sms() * kBBlocksPerSM;
  int64_t slen = 1, zlen = 1;
  for (int b = 0; b < count; b++) {
    int64_t N = 1, nmin = d[b].dims[0];
    for (int m = 0; m < d[b].order; m++) {
      N *= d[b].dims[m];
      nmin = std::min(nmin, d[b].dims[m]);
      zlen = std::max(zlen, d[b].dims[m]);
    }
    slen = std::max(slen, N / nmin);
  }
  L.slen = align_up((size_t)slen, 64);
  L.zlen = align_up((size_t)zlen, 64);
  L.off_counter = 0;
  L.off_items = 256;
  L.off_scratch = L.off_items + align_up((size_t)count * sizeof(HItem), 256);
  L.total = L.off_scratch + (size_t)L.blocks * (3 * L.slen + L.zlen) * sizeof(float);
  return L;
}

tvc_status check_tvc_descs(const tvc_batch_desc* d, int count, std::vector<BItem>* items) {
  std::vector<std::pair<int64_t, int>> order;
  for (int b = 0; b < count; b++) {
    Shape s;
    if (make_shape(d[b].order, d[b].dims, d[b].mode, &s) != TVC_OK) return TVC_ERR_INVALID_ARG;
    if (!d[b].A) return TVC_ERR_INVALID_ARG;
    if (d[b].y && !d[b].x) return TVC_ERR_INVALID_ARG;
    if ((d[b].gx || d[b].gA) && !d[b].gy) return TVC_ERR_INVALID_ARG;
    if (d[b].gA && !d[b].x) return TVC_ERR_INVALID_ARG;
    order.push_back({s.N, b});
  }
  std::stable_sort(order.begin(), order.end(), [](auto& a, auto& b) { return a.first > b.first; });
  if (items) {
    items->clear();
    for (auto& pr : order) {
      const tvc_batch_desc& e = d[pr.second];
      Shape s;
      make_shape(e.order, e.dims, e.mode, &s);
      BItem it{};
      it.A = e.A;
      it.x = e.x;
      it.y = e.y;
      it.gy = e.gy;
      it.gx = e.gx;
      it.gA = e.gA;
      it.u = s.u;
      it.nk = s.nk;
      it.v = s.v;
      it.gf = pick_G(s.nk, s.v);
      it.gxk = 0;
      it.gxp = 0;
      items->push_back(it);
    }
  }
  return TVC_OK;
}

}  // namespace
}  // namespace tvcg

using namespace tvcg;

extern "C" size_t tvc_batched_workspace_size(const tvc_batch_desc* descs, int count) {
  if (count < 0 || (count > 0 && !descs)) return 0;
  std::vector<BItem> items;
  if (check_tvc_descs(descs, count, &items) != TVC_OK) return 0;
  std::vector<WItem> work;
  make_work(items, &work);
  return layout_tvc_items(items, work.size()).total;
}

extern "C" tvc_status tvc_batched(const tvc_batch_desc* descs, int count, int flags, void* workspace, size_t ws_bytes,
                                  tvc_stream_t stream) {
  if (count < 0 || !descs) return TVC_ERR_INVALID_ARG;
  if (count == 0) return TVC_OK;
  std::vector<BItem> items;
  tvc_status rc = check_tvc_descs(descs, count, &items);
  if (rc != TVC_OK) return rc;
  std::vector<WItem> work;
  make_work(items, &work);
  const BLayout L = layout_tvc_items(items, work.size());
  if (!workspace || ws_bytes < L.total) return TVC_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  char* w = static_cast<char*>(workspace);
  int* hdr = reinterpret_cast<int*>(w + L.off_counter);
  if (!(flags & TVC_BATCH_PREUPLOADED)) {
    const int nwork = (int)work.size();
    if (cudaMemcpyAsync(w + L.off_items, items.data(), items.size() * sizeof(BItem), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(w + L.off_scratch, work.data(), work.size() * sizeof(WItem), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(hdr + 1, &nwork, sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        // per-tensor gx counters: zero now; the last item of a tensor resets its own
        cudaMemsetAsync(w + L.off_gxcnt, 0, items.size() * sizeof(int), st) != cudaSuccess)
      return TVC_ERR_CUDA;
    // The host vectors die here: wait for the copies (pageable sources).
    if (cudaStreamSynchronize(st) != cudaSuccess) return TVC_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_nwork[workspace] = nwork;
  }
  int nwork = 0;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto itn = g_nwork.find(workspace);
    if (itn == g_nwork.end()) return TVC_ERR_INVALID_ARG;  // PREUPLOADED without a prior upload
    nwork = itn->second;
  }
  cudaMemsetAsync(hdr, 0, sizeof(int), st);
  tvc_batched_kernel<<<L.blocks, kBBT, 0, st>>>(reinterpret_cast<const BItem*>(w + L.off_items),
                                               reinterpret_cast<const WItem*>(w + L.off_scratch), nwork, hdr,
                                               reinterpret_cast<int*>(w + L.off_gxcnt),
                                               reinterpret_cast<float*>(w + L.off_gxpart));
  count_launches(1);
  return cuda_status(cudaGetLastError());
}

extern "C" tvc_status tvc_batched_autotune(const tvc_batch_desc* descs, int count, void* workspace, size_t ws_bytes,
                                           tvc_stream_t stream) {
  // Times the candidate lane counts of the forward contraction on the
  // tensors of every shape class and records the fastest; synchronises.
  if (count <= 0 || !descs) return TVC_ERR_INVALID_ARG;
  std::vector<BItem> items;
  tvc_status rc = check_tvc_descs(descs, count, &items);
  if (rc != TVC_OK) return rc;
  std::vector<WItem> allwork;
  make_work(items, &allwork);
  const BLayout L = layout_tvc_items(items, allwork.size());
  if (!workspace || ws_bytes < L.total) return TVC_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  char* w = static_cast<char*>(workspace);
  // every shape class of forward rows (v == 1, where lanes split a row)
  // with the tensors that belong to it
  std::map<std::pair<int, int>, std::vector<BItem>> classes;
  for (const BItem& it : items) {
    if (!it.y || it.v != 1) continue;
    BItem one = it;
    one.gx = nullptr;
    one.gA = nullptr;
    classes[{(int)clog2(it.v), (int)clog2(it.nk)}].push_back(one);
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int cands[5] = {1, 4, 8, 16, 32};
  for (auto& kv : classes) {
    std::vector<BItem> sub = kv.second;  // at most 256 tensors of the class
    if (sub.size() > 256) sub.resize(256);
    float best = 1e30f;
    int bestG = rule_G(sub[0].nk, sub[0].v);
    for (int G : cands) {
      for (BItem& it : sub) it.gf = G;
      std::vector<WItem> wk;
      make_work(sub, &wk);
      cudaMemcpy(w + L.off_items, sub.data(), sub.size() * sizeof(BItem), cudaMemcpyHostToDevice);
      cudaMemcpy(w + L.off_scratch, wk.data(), wk.size() * sizeof(WItem), cudaMemcpyHostToDevice);
      float tot = 0.0f;
      for (int rep = 0; rep < 3; rep++) {
        cudaMemsetAsync(w + L.off_counter, 0, sizeof(int), st);
        cudaEventRecord(e0, st);
        tvc_batched_kernel<<<L.blocks, kBBT, 0, st>>>(reinterpret_cast<const BItem*>(w + L.off_items),
                                                     reinterpret_cast<const WItem*>(w + L.off_scratch),
                                                     (int)wk.size(), reinterpret_cast<int*>(w + L.off_counter),
                                                     reinterpret_cast<int*>(w + L.off_gxcnt),
                                                     reinterpret_cast<float*>(w + L.off_gxpart));
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) tot += ms;
      }
      count_launches(3);
      if (tot < best) {
        best = tot;
        bestG = G;
      }
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[kv.first] = bestG;
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_nwork.erase(workspace);  // the workspace no longer holds an uploaded batch
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return cuda_status(cudaGetLastError());
}

extern "C" size_t hopm_batched_workspace_size(const hopm_batch_desc* descs, int count) {
  if (count < 0 || (count > 0 && !descs)) return 0;
  for (int b = 0; b < count; b++)
    if (descs[b].order < 2 || check_dims(descs[b].order, descs[b].dims, nullptr) != TVC_OK) return 0;
  return layout_hopm(descs, count).total;
}

extern "C" tvc_status hopm_batched(const hopm_batch_desc* descs, int count, int iters, int flags, void* workspace,
                                   size_t ws_bytes, tvc_stream_t stream) {
  if (count < 0 || iters < 0 || !descs) return TVC_ERR_INVALID_ARG;
  if (count == 0) return TVC_OK;
  for (int b = 0; b < count; b++) {
    if (descs[b].order < 2 || !descs[b].A || check_dims(descs[b].order, descs[b].dims, nullptr) != TVC_OK)
      return TVC_ERR_INVALID_ARG;
    for (int m = 0; m < descs[b].order; m++)
      if (!descs[b].x[m]) return TVC_ERR_INVALID_ARG;
  }
  const BLayout L = layout_hopm(descs, count);
  if (!workspace || ws_bytes < L.total) return TVC_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  char* w = static_cast<char*>(workspace);
  if (!(flags & TVC_BATCH_PREUPLOADED)) {
    std::vector<std::pair<int64_t, int>> order;
    for (int b = 0; b < count; b++) {
      int64_t N = 1;
      for (int m = 0; m < descs[b].order; m++) N *= descs[b].dims[m];
      order.push_back({N, b});
    }
    std::stable_sort(order.begin(), order.end(), [](auto& a, auto& b) { return a.first > b.first; });
    std::vector<HItem> items;
    for (auto& pr : order) {
      const hopm_batch_desc& e = descs[pr.second];
      HItem it{};
      it.A = e.A;
      it.d = e.order;
      for (int m = 0; m < e.order; m++) {
        it.dims[m] = e.dims[m];
        it.x[m] = e.x[m];
      }
      // lanes per output of the two big contractions (A x_1 x_1, A x_0 x_0)
      int64_t N = 1;
      for (int m = 0; m < e.order; m++) N *= e.dims[m];
      it.gsel[0] = pick_G(e.dims[0], N / e.dims[0]);
      it.gsel[1] = pick_G(e.dims[1], N / (e.dims[0] * e.dims[1]));
      it.lam = e.lambda_out;
      it.status = e.status_out;
      items.push_back(it);
    }
    if (cudaMemcpyAsync(w + L.off_items, items.data(), items.size() * sizeof(HItem), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      return TVC_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return TVC_ERR_CUDA;
  }
  cudaMemsetAsync(w + L.off_counter, 0, sizeof(int), st);
  hopm_batched_kernel<<<L.blocks, kBBT, 0, st>>>(reinterpret_cast<const HItem*>(w + L.off_items), count, iters,
                                                reinterpret_cast<int*>(w + L.off_counter),
                                                reinterpret_cast<float*>(w + L.off_scratch), L.slen, L.zlen);
  count_launches(1);
  return cuda_status(cudaGetLastError());
}
