// search_common.cuh -- device helpers shared by the wave kernels (search.cu),
// the compile-time-planned kernels and the persistent kernel (search_fixed.cu).
#pragma once
#include <float.h>
#include <limits.h>
#include <math.h>

#include "common.cuh"
#include "prnu.h"

namespace prnu {

// ---------------------------------------------------------------- helpers

struct WarpRed {
  float ma;
  int ia;
  float mb;
  int ib;
  double sa;
  double sb;
};

__device__ __forceinline__ void better_f(float& v, int& i, float v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) {
    v = v2;
    i = i2;
  }
}
__device__ __forceinline__ void better_d(double& v, int& i, double v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) {
    v = v2;
    i = i2;
  }
}
__device__ __forceinline__ void warp_maxarg(float& v, int& i) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    float v2 = __shfl_xor_sync(0xffffffffu, v, o);
    int i2 = __shfl_xor_sync(0xffffffffu, i, o);
    better_f(v, i, v2, i2);
  }
}
__device__ __forceinline__ void warp_maxarg_d(double& v, int& i) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    int i2 = __shfl_xor_sync(0xffffffffu, i, o);
    better_d(v, i, v2, i2);
  }
}

// The best candidate of group g (one frame and fingerprint), by one warp
// (lane = its lane): the highest PCE, the lowest index among equal ones
// (candidates gstart[f] + (g - f*share) + k*share of frame f = g / share),
// its (lam, theta), cyclic peak as a signed shift, PCE and peak, into out[g].
__device__ __forceinline__ void argmax_group(const CandResult* __restrict__ res, const WorkItem* __restrict__ items,
                                             const int* __restrict__ gstart, int share, prnu_result* out, int H,
                                             int W, int g, int lane) {
  const int f = g / share;
  const int b = gstart[f] + (g - f * share), n = (gstart[f + 1] - gstart[f]) / share;
  double bv = -INFINITY;
  int bi = INT_MAX;
  for (int k = lane; k < n; k += 32) {
    const int i = b + k * share;
    better_d(bv, bi, res[i].pce, i);
  }
  warp_maxarg_d(bv, bi);
  if (lane == 0) {
    prnu_result r;
    if (bi == INT_MAX || n == 0) {
      r.lam = 0.f; r.th_deg = 0.f; r.dy = 0; r.dx = 0; r.pce = 0.0; r.peak = 0.f; r.cand_idx = -1;
    } else {
      const CandResult c = res[bi];
      const WorkItem it = items[bi];
      r.lam = it.lam;
      r.th_deg = it.th_deg;
      r.dy = c.py < (H + 1) / 2 ? c.py : c.py - H;
      r.dx = c.px < (W + 1) / 2 ? c.px : c.px - W;
      if (2 * c.py == H) r.dy = -H / 2;
      if (2 * c.px == W) r.dx = -W / 2;
      r.pce = c.pce;
      r.peak = c.peak;
      r.cand_idx = c.cand;
    }
    out[g] = r;
  }
}
__device__ __forceinline__ double warp_sum(double s) {
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Compensated FP32 summation (Knuth's TwoSum): the pair (s, c) holds the
// value s + c; adding b keeps the rounding error of s + b in c.
__device__ __forceinline__ void csum_add(float& s, float& c, float b) {
  const float t = s + b;
  const float bp = t - s;
  const float e = (s - (t - bp)) + (b - bp);
  s = t;
  c += e;
}
__device__ __forceinline__ void warp_csum(float& s, float& c) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
    c += c2;
    csum_add(s, c, s2);
  }
}

// Per-warp partial statistics of a row pair (rows a and b).
struct RowRed {
  float ma;
  int ia;
  float mb;
  int ib;
  float sa, ca, sb, cb;   // compensated sums of squares
};
static_assert(sizeof(RowRed) == sizeof(WarpRed), "row reductions share the WarpRed scratch");

// Reduce the per-thread row statistics of a row pair to one RowRed per warp
// (lane 0 writes red[warp]).  Per thread: FP32 partial over its few elements;
// across the warp: compensated FP32.
__device__ __forceinline__ void row_stats_warp(float ma, int ia, float mb, int ib, float sa, float sb, int t,
                                               RowRed* red) {
  float ca = 0.f, cb = 0.f;
  warp_maxarg(ma, ia);
  warp_maxarg(mb, ib);
  warp_csum(sa, ca);
  warp_csum(sb, cb);
  if ((t & 31) == 0) red[t >> 5] = RowRed{ma, ia, mb, ib, sa, ca, sb, cb};
}
// Order-preserving map of a float to a signed int (for max reductions on
// integer units): x < y  <=>  key(x) < key(y) for non-NaN x, y; -0 and +0 both
// map to 0, as they compare equal.
__device__ __forceinline__ int float_key(float v) {
  const int i = __float_as_int(v);
  return i >= 0 ? i : (i == INT_MIN ? 0 : i ^ 0x7fffffff);
}
__device__ __forceinline__ float key_float(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

// Combine nw warps' RowRed (after a barrier) into the two rows' statistics.
__device__ __forceinline__ void row_stats_final(const RowRed* red, int nw, RowStat* st) {
  RowRed r = red[0];
#pragma unroll 1
  for (int k = 1; k < nw; ++k) {
    const RowRed q = red[k];
    better_f(r.ma, r.ia, q.ma, q.ia);
    better_f(r.mb, r.ib, q.mb, q.ib);
    r.ca += q.ca;
    csum_add(r.sa, r.ca, q.sa);
    r.cb += q.cb;
    csum_add(r.sb, r.cb, q.sb);
  }
  st[0] = RowStat{r.ma, r.ia, (double)r.sa + (double)r.ca};
  st[1] = RowStat{r.mb, r.ib, (double)r.sb + (double)r.cb};
}
// cyclic distance between indices a and b modulo n
__device__ __forceinline__ int cdist(int a, int b, int n) {
  int d = a - b;
  if (d < 0) d = -d;
  return d < n - d ? d : n - d;
}

constexpr int kHalfWindow = 5;      // Eq. 3: 11 x 11 exclusion
constexpr int kWindowCount = 121;

// Bilinear sample of an H x W frame (row pitch `pitch`, pixel (0, 0) at
// element `base` of R) at (qx, qy); each tap outside the frame contributes 0.
template <int DT>
__device__ __forceinline__ float bilinear(const void* R, size_t base, int H, int W, int pitch, float qx, float qy) {
  const float fx0 = floorf(qx), fy0 = floorf(qy);
  const float fx = qx - fx0, fy = qy - fy0;
  const int x0 = (int)fx0, y0 = (int)fy0;
  const bool xi0 = (unsigned)x0 < (unsigned)W, xi1 = (unsigned)(x0 + 1) < (unsigned)W;
  const bool yi0 = (unsigned)y0 < (unsigned)H, yi1 = (unsigned)(y0 + 1) < (unsigned)H;
  const size_t r0 = base + (size_t)((long long)y0 * pitch + x0);
  const float v00 = (yi0 && xi0) ? load_store_type<DT>(R, r0) : 0.f;
  const float v01 = (yi0 && xi1) ? load_store_type<DT>(R, r0 + 1) : 0.f;
  const float v10 = (yi1 && xi0) ? load_store_type<DT>(R, r0 + pitch) : 0.f;
  const float v11 = (yi1 && xi1) ? load_store_type<DT>(R, r0 + pitch + 1) : 0.f;
  const float gx = 1.f - fx, gy = 1.f - fy;
  return gy * (gx * v00 + fx * v01) + fy * (gx * v10 + fx * v11);
}

template <int DT>
struct StoreT;
template <>
struct StoreT<kF32> {
  using type = float;
  __device__ __forceinline__ static float ld(const float* p) { return __ldg(p); }
};
template <>
struct StoreT<kF16> {
  using type = __half;
  __device__ __forceinline__ static float ld(const __half* p) { return __half2float(__ldg(p)); }
};
template <>
struct StoreT<kBF16> {
  using type = __nv_bfloat16;
  __device__ __forceinline__ static float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
};
// pair layouts: one load gives two horizontally adjacent taps
template <>
struct StoreT<kF16P> {
  using type = __half2;
  __device__ __forceinline__ static float2 ld2(const __half2* p) { return __half22float2(__ldg(p)); }
};
template <>
struct StoreT<kBF16P> {
  using type = __nv_bfloat162;
  __device__ __forceinline__ static float2 ld2(const __nv_bfloat162* p) { return __bfloat1622float2(__ldg(p)); }
};
template <int DT>
constexpr bool kPairStore = DT == kF16P || DT == kBF16P;

// Zero-bordered frame layout read by the compile-time-planned kernels: one
// zero row/column before the frame and two after it, row pitch W + 3, so
// that every clamped bilinear tap is a valid address.
__host__ __device__ constexpr int pad_pitch(int W) { return W + 3; }
__host__ __device__ constexpr size_t pad_frame_elems(int H, int W) { return (size_t)(H + 3) * (W + 3); }
__host__ __device__ constexpr size_t pad_origin(int W) { return (size_t)(W + 3) + 1; }

// bilinear<DT> on the zero-bordered layout, W a compile-time constant, `fr`
// pointing at pixel (0, 0).  With CLAMP the sample point is clamped to
// [-1, W] x [-1, H]: inside that box the taps and weights are those of
// bilinear<DT> (a tap in the border reads 0); outside it every tap of
// bilinear<DT> is outside the frame, and the clamped point puts weight 1 on a
// border zero and weight 0 on the rest.  So the value is the same, with no
// predicate: one index, four loads at fixed offsets.  Without CLAMP the
// caller guarantees the point is in the box.  The tap index fy0*P + fx0 is
// formed in float, where it is exact (|value| < 2^24 for the frame sizes here).
template <int DT, int W, bool CLAMP = true>
__device__ __forceinline__ float bilinear_pad(const typename StoreT<DT>::type* __restrict__ fr, int H, float qx,
                                              float qy) {
  using S = StoreT<DT>;
  constexpr int P = pad_pitch(W);
  if constexpr (CLAMP) {
    qx = fminf(fmaxf(qx, -1.f), (float)W);
    qy = fminf(fmaxf(qy, -1.f), (float)H);
  }
  const float fx0 = floorf(qx), fy0 = floorf(qy);
  const float fx = qx - fx0, fy = qy - fy0;
  const auto* p = fr + __float2int_rn(fmaf(fy0, (float)P, fx0));
  float v00, v01, v10, v11;
  if constexpr (kPairStore<DT>) {
    const float2 a = S::ld2(p), b = S::ld2(p + P);
    v00 = a.x;
    v01 = a.y;
    v10 = b.x;
    v11 = b.y;
  } else {
    v00 = S::ld(p);
    v01 = S::ld(p + 1);
    v10 = S::ld(p + P);
    v11 = S::ld(p + P + 1);
  }
  const float top = fmaf(fx, v01 - v00, v00), bot = fmaf(fx, v11 - v10, v10);
  return fmaf(fy, bot - top, top);
}

// Loads of data that other blocks of the same launch may have written (the
// persistent kernel reuses workspace slots): cached in L2 only, never in the
// non-coherent L1.
__device__ __forceinline__ float2 ld_l2(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ RowStat ld_l2(const RowStat* p) {
  RowStat r;
  const float2 a = __ldcg(reinterpret_cast<const float2*>(p));
  r.max = a.x;
  r.arg = __float_as_int(a.y);
  r.sumsq = __ldcg(&p->sumsq);
  return r;
}

// Full spectrum z = G_a + i G_b of two packed half-spectrum rows (the inverse
// of the split done after the forward row FFT).
__device__ __forceinline__ void build_full_row(float2* buf, const float2* __restrict__ pa,
                                               const float2* __restrict__ pb, int W, int t, int T) {
  const int Wh = W >> 1;
  for (int k = t; k < Wh; k += T) {
    const float2 A = pa[k], B = pb[k];
    if (k == 0) {
      buf[rpad(0)] = make_float2(A.x, B.x);
      buf[rpad(Wh)] = make_float2(A.y, B.y);
    } else {
      buf[rpad(k)] = make_float2(A.x - B.y, A.y + B.x);
      buf[rpad(W - k)] = make_float2(A.x + B.y, B.x - A.y);
    }
  }
}

__host__ __device__ inline size_t row_smem_bytes(int W, int ppb) {
  return (size_t)ppb * 2 * row_smem_len(W) * sizeof(float2) + (size_t)ppb * 32 * sizeof(WarpRed);
}

// Peak, energy outside the cyclic 11x11 window and PCE (Eq. 3) of candidate
// `is` whose row statistics and spectrum sit in workspace slot `ws`; all
// threads of the block take part (any block size that is a multiple of 32).
static __device__ __noinline__ void finalize_body(const PassArgs& a, int is, int ws, float2* smem) {
  __shared__ int s_py, s_px;
  __shared__ float s_peak;
  const int T = blockDim.x, t = threadIdx.x;
  const int H = a.H, W = a.W, Wh = W >> 1;
  const WorkItem it = item_of(a, is);
  const RowStat* st = a.stats + (size_t)ws * H;
  const float2* Z = a.spec + (size_t)ws * H * Wh;
  float2* const bufA = smem;
  float2* const bufB = smem + row_smem_len(W);
  WarpRed* red = reinterpret_cast<WarpRed*>(smem + 2 * row_smem_len(W));
  const int nw = T >> 5, w = t >> 5;

  float bv = -INFINITY;
  int bi = INT_MAX;
  for (int y = t; y < H; y += T) {
    const RowStat r = st[y];
    better_f(bv, bi, r.max, y * W + r.arg);
  }
  warp_maxarg(bv, bi);
  if ((t & 31) == 0) { red[w].ma = bv; red[w].ia = bi; }
  __syncthreads();
  if (t == 0) {
    for (int k = 1; k < nw; ++k) better_f(bv, bi, red[k].ma, red[k].ia);
    if (bi == INT_MAX) bi = 0;
    s_peak = bv;
    s_py = bi / W;
    s_px = bi - (bi / W) * W;
  }
  __syncthreads();
  const int py = s_py, px = s_px;
  double e = 0.0;
  for (int y = t; y < H; y += T)
    if (cdist(y, py, H) > kHalfWindow) e += st[y].sumsq;
  int prev = -1;
  for (int d = -kHalfWindow; d <= kHalfWindow; ++d) {
    const int r = (py + d + H) % H;
    const int p = r >> 1;
    if (p == prev) continue;
    prev = p;
    build_full_row(bufA, Z + (size_t)(2 * p) * Wh, Z + (size_t)(2 * p + 1) * Wh, W, t, T);
    __syncthreads();
    const float2* buf = fft_row<true>(bufA, bufB, a.prow, a.tw, t, T);
    for (int q = 0; q < 2; ++q) {
      if (cdist(2 * p + q, py, H) > kHalfWindow) continue;
      for (int x = t; x < W; x += T) {
        if (cdist(x, px, W) <= kHalfWindow) continue;
        const float2 v = buf[rpad(x)];
        const double c = q ? v.y : v.x;
        e += c * c;
      }
    }
    __syncthreads();
  }
  e = warp_sum(e);
  if ((t & 31) == 0) red[w].sa = e;
  __syncthreads();
  if (t == 0) {
    double etot = red[0].sa;
    for (int k = 1; k < nw; ++k) etot += red[k].sa;
    const double E = etot / ((double)H * (double)W - (double)kWindowCount);
    const double pk = (double)s_peak;
    double pce;
    if (E > 0.0) pce = (pk < 0 ? -1.0 : 1.0) * pk * pk / E;
    else pce = pk == 0.0 ? 0.0 : (pk < 0 ? -INFINITY : INFINITY);
    const FpDesc fp = a.fps[it.fp];
    double pv = pk / ((double)H * (double)W) * (double)(*fp.inv_scale);
    if (a.scale) pv /= (double)a.scale[it.frame];
    CandResult r;
    r.pce = pce;
    r.peak = (float)pv;
    r.py = py;
    r.px = px;
    r.cand = it.cand;
    r.group = it.group;
    r.pad = 0;
    *result_of(a, is) = r;
  }
}


}  // namespace prnu
