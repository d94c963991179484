// Batched contractions, adjoints and power methods over many independent
// FP32 tensors of uneven order and shape, each batch in one persistent
// launch (the GPU counterpart of the paper's task-based execution, Section
// 4.3, where many TVCs overlap instead of joining after each one).
//
// The host uploads one descriptor per tensor (largest first) into the
// workspace; a persistent kernel of a few blocks per SM then pulls tensors
// from an atomic work counter, and one block runs all the work of its
// tensor (forward TVC, gx, gA; or every sweep of a HOPM) with block-level
// routines.  With TVC_BATCH_PREUPLOADED the descriptors of a previous call
// are reused and a call issues only a memset and one kernel, so it can be
// captured in a CUDA graph and replayed.
//
// Block-level contraction: a group of G lanes (G a power of two <= 32)
// computes one output, its lanes splitting the contracted index; G = 1 is
// one thread per output (coalesced when v is large), G = 32 a warp per
// output (coalesced along rows when v == 1).  The autotuner picks G per
// shape class (v and n_k rounded to powers of two) by timing the
// candidates; untuned classes use a fixed rule.
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
  int gf, gb;  // lanes per output: forward contraction, gx
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

// gx[j] = sum_{i,l} A[(i*nk + j)*v + l] gy[i*v + l]; a group of G lanes per j.
// Compensated FP32 sums (the reduction can be long).
__device__ void blk_gx(const float* __restrict__ A, int64_t u, int64_t nk, int64_t v, const float* __restrict__ gy,
                       float* __restrict__ gx, int G, int64_t j_begin = 0, int64_t j_end = -1) {
  const int lane = threadIdx.x & 31;
  const int p = lane & (G - 1);
  const int gw = 32 / G;
  const int64_t je = (j_end < 0) ? nk : j_end;
  const int64_t ngroups = (int64_t)(kBBT / 32) * gw;
  for (int64_t base = j_begin + (int64_t)(threadIdx.x >> 5) * gw; base < je; base += ngroups) {
    const int64_t j = base + lane / G;
    KahanF32 acc;
    if (j < je) {
      if (v >= G) {
        for (int64_t i = 0; i < u; i++) {
          const float* a = A + (i * nk + j) * v;
          const float* g = gy + i * v;
          float part = 0.0f;
          for (int64_t l = p; l < v; l += 8 * G) {  // eight predicated loads in flight
            float av[8], gv[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
              const bool ok = l + q * G < v;
              av[q] = ok ? __ldcs(a + l + q * G) : 0.0f;
              gv[q] = ok ? __ldg(g + l + q * G) : 0.0f;
            }
#pragma unroll
            for (int q = 0; q < 8; q++) part = __fmaf_rn(av[q], gv[q], part);
          }
          acc.add(part);
        }
      } else {
        // v < G: lanes split the slabs i, eight slabs in flight per lane
        for (int64_t i = p; i < u; i += 8 * G) {
          for (int64_t l = 0; l < v; l++) {
            float av[8], gv[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
              const int64_t ii = i + q * G;
              const bool ok = ii < u;
              av[q] = ok ? __ldcs(A + (ii * nk + j) * v + l) : 0.0f;
              gv[q] = ok ? __ldg(gy + ii * v + l) : 0.0f;
            }
            float part = 0.0f;
#pragma unroll
            for (int q = 0; q < 8; q++) part = __fmaf_rn(av[q], gv[q], part);
            acc.add(part);
          }
        }
      }
    }
    float t = acc.value();
    for (int off = G / 2; off > 0; off >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, off);
    if (j < je && p == 0) gx[j] = t;
  }
}

// gx[j] for a few j (<= 8) with all 256 threads: a team of T = 256/J
// threads (whole warps) per j splits the (i, l) space (lane t: l = t % v'
// and i = t / v' with v' = min(v, T), stepping by T / v'), compensated sums,
// then warp shuffles and a fixed-order sum of the team's warps.
__device__ void blk_gx_teams(const float* __restrict__ A, int64_t u, int64_t nk, int64_t v,
                             const float* __restrict__ gy, float* __restrict__ gx, int64_t j_begin, int64_t j_end,
                             float* red /* shared, kBBT/32 floats */) {
  const int J = (int)(j_end - j_begin);
  int T = 256;
  while (T > 32 && T * J > 256) T >>= 1;
  const int team = threadIdx.x / T, t = threadIdx.x % T;
  const int64_t j = j_begin + team;
  const int64_t vv = v < T ? v : T;
  const int lanes = (int)((T / vv) * vv);
  KahanF32 acc;
  if (team < J && t < lanes) {
    const int64_t l0 = t % vv, i0 = t / vv, istep = T / vv;
    for (int64_t i = i0; i < u; i += istep) {
      const float* a = A + (i * nk + j) * v;
      const float* g = gy + i * v;
      float part = 0.0f;
      for (int64_t l = l0; l < v; l += 8 * vv) {
        float av[8], gv[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const bool ok = l + q * vv < v;
          av[q] = ok ? __ldcs(a + l + q * vv) : 0.0f;
          gv[q] = ok ? __ldg(g + l + q * vv) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 8; q++) part = __fmaf_rn(av[q], gv[q], part);
      }
      acc.add(part);
    }
  }
  float s = acc.value();
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (t == 0 && team < J) {
    float tot = 0.0f;
    for (int w = 0; w < T / 32; w++) tot += red[team * (T / 32) + w];
    gx[j] = tot;
  }
  __syncthreads();
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
// 1 = gx[j] for j in [a0, a1), 2 = gA over slabs [a0, a1) and rows [c0, c1).
struct WItem {
  int b, kind;
  int64_t a0, a1, c0, c1;
};

__global__ void __launch_bounds__(kBBT, 6) tvc_batched_kernel(const BItem* __restrict__ items,
                                                           const WItem* __restrict__ work, int nwork, int* counter) {
  __shared__ int slot;
  __shared__ float red[kBBT / 32];
  for (int w = grab(counter, &slot); w < nwork; w = grab(counter, &slot)) {
    const WItem wi = work[w];
    const BItem it = items[wi.b];
    if (wi.kind == 0)
      blk_tvc(it.A, it.u, it.nk, it.v, it.x, it.y, it.gf, wi.a0, wi.a1);
    else if (wi.kind == 1) {
      if (wi.a1 - wi.a0 <= 8)
        blk_gx_teams(it.A, it.u, it.nk, it.v, it.gy, it.gx, wi.a0, wi.a1, red);
      else
        blk_gx(it.A, it.u, it.nk, it.v, it.gy, it.gx, it.gb, wi.a0, wi.a1);
    }
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
            blk_tvc(it.A, n[0], n[1], rest2, it.x[1], S1, it.gsel[1]);  // T = A x_1 x_1
          else
            blk_tvc(it.A, 1, n[0], N / n[0], it.x[0], S1, it.gsel[0]);  // W_1 = A x_0 x_0
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

// Autotuner cache: (kind, log2 v, log2 n_k) -> G.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tune;
std::map<void*, int> g_nwork;  // work items uploaded per workspace

int rule_G(int kind, int64_t nk, int64_t v) {
  if (kind == 0) {  // forward: lanes split n_k
    if (v >= 32) return 1;
    if (v >= 8) return 4;
    return nk >= 64 ? 32 : 8;
  }
  // gx: lanes split the (i, l) columns (for v < 8 the slabs i)
  return v >= 32 ? 32 : 8;
}

int pick_G(int kind, int64_t nk, int64_t v) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find({kind, (int)clog2(v), (int)clog2(nk)});
  return it != g_tune.end() ? it->second : rule_G(kind, nk, v);
}

struct BLayout {
  size_t off_counter = 0, off_items = 0, off_scratch = 0, total = 0;
  int64_t slen = 0, zlen = 0;
  int blocks = 0;
};

// Work of about this many elements per item (a few MB): large tensors
// spread over many blocks, small ones make a single item.
constexpr int64_t kItemElems = 1 << 20;

int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

void make_work(const std::vector<BItem>& items, std::vector<WItem>* work) {
  work->clear();
  for (int b = 0; b < (int)items.size(); b++) {
    const BItem& it = items[b];
    const int64_t uv = it.u * it.v, N = uv * it.nk;
    if (it.y) {
      const int64_t per = std::max<int64_t>(256, cdiv64(kItemElems, it.nk) / 256 * 256);
      for (int64_t o = 0; o < uv; o += per) work->push_back({b, 0, o, std::min(uv, o + per), 0, 0});
    }
    if (it.gx) {
      const int64_t per = std::max<int64_t>(1, kItemElems / std::max<int64_t>(1, uv));
      for (int64_t j = 0; j < it.nk; j += per) work->push_back({b, 1, j, std::min(it.nk, j + per), 0, 0});
    }
    if (it.gA) {
      const int64_t S = it.nk * it.v;
      if (it.v >= 32) {
        // rectangles of slabs x rows
        const int64_t rows = std::max<int64_t>(1, std::min<int64_t>(it.nk, kItemElems / it.v));
        const int64_t slabs = std::max<int64_t>(1, kItemElems / (rows * it.v));
        for (int64_t i = 0; i < it.u; i += slabs)
          for (int64_t j = 0; j < it.nk; j += rows)
            work->push_back({b, 2, i, std::min(it.u, i + slabs), j, std::min(it.nk, j + rows)});
      } else {
        const int64_t slabs = std::max<int64_t>(1, kItemElems / S);
        for (int64_t i = 0; i < it.u; i += slabs) work->push_back({b, 2, i, std::min(it.u, i + slabs), 0, it.nk});
      }
    }
    (void)N;
  }
}

// Workspace of a tensor batch: header, descriptors, work items (the exact
// count, from the same construction the call uses).
tvc_status check_tvc_descs(const tvc_batch_desc* d, int count, std::vector<BItem>* items);

BLayout layout_tvc_items(const std::vector<BItem>& items, size_t nwork) {
  BLayout L;
  L.off_counter = 0;
  L.off_items = 256;
  L.off_scratch = L.off_items + align_up(items.size() * sizeof(BItem), 256);
  L.total = L.off_scratch + align_up(nwork * sizeof(WItem), 256);
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
      it.gf = pick_G(0, s.nk, s.v);
      it.gb = pick_G(1, s.nk, s.v);
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
        cudaMemcpyAsync(hdr + 1, &nwork, sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
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
                                               reinterpret_cast<const WItem*>(w + L.off_scratch), nwork, hdr);
  count_launches(1);
  return cuda_status(cudaGetLastError());
}

extern "C" tvc_status tvc_batched_autotune(const tvc_batch_desc* descs, int count, void* workspace, size_t ws_bytes,
                                           tvc_stream_t stream) {
  // Times the candidate lane counts on one tensor of every shape class
  // (forward contraction and gx) and records the fastest; synchronises.
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
  // every shape class with the tensors that belong to it (forward, gx)
  std::map<std::tuple<int, int, int>, std::vector<BItem>> classes;
  for (const BItem& it : items)
    for (int kind = 0; kind < 2; kind++) {
      if (kind == 0 && !it.y) continue;
      if (kind == 1 && !it.gx) continue;
      BItem one = it;
      one.y = kind == 0 ? it.y : nullptr;
      one.gx = kind == 1 ? it.gx : nullptr;
      one.gA = nullptr;
      classes[std::make_tuple(kind, (int)clog2(it.v), (int)clog2(it.nk))].push_back(one);
    }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int cands[5] = {1, 4, 8, 16, 32};
  for (auto& kv : classes) {
    const int kind = std::get<0>(kv.first);
    std::vector<BItem> sub = kv.second;  // at most 256 tensors of the class
    if (sub.size() > 256) sub.resize(256);
    float best = 1e30f;
    int bestG = rule_G(kind, sub[0].nk, sub[0].v);
    for (int G : cands) {
      for (BItem& it : sub) (kind == 0 ? it.gf : it.gb) = G;
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
                                                     (int)wk.size(), reinterpret_cast<int*>(w + L.off_counter));
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
      it.gsel[0] = pick_G(0, e.dims[0], N / e.dims[0]);
      it.gsel[1] = pick_G(0, e.dims[1], N / (e.dims[0] * e.dims[1]));
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
