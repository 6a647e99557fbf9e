// search.cu -- kernels of the EIS-inversion grid search (Sec. 3.2) and their launchers.
//
// Per candidate (frame f, fingerprint p, grid node (lambda, theta)) the fused
// path runs four kernels over a wave of candidates:
//   k_row_forward : inverse warp of the residual (Eq. 4, bilinear, zero
//                   outside) fused with the row FFT; two real rows share one
//                   complex FFT; output is the packed half spectrum
//                   [H][W/2] complex whose column 0 holds (DC, Nyquist) pairs;
//   k_col         : column FFT, product conj(X^) K0^ with the cached
//                   fingerprint spectrum, inverse column FFT, in place;
//   k_row_inverse : inverse row FFT (two rows per complex FFT) and per-row
//                   max / first arg-max / sum of squares of C;
//   k_finalize    : peak over rows, energy outside the cyclic 11x11 window
//                   (the window's rows are recomputed from the spectrum) and
//                   PCE (Eq. 3).
// k_argmax then keeps the best candidate of each (frame, fingerprint).
#include <float.h>
#include <limits.h>
#include <math.h>

#include <algorithm>

#include "internal.h"
#include "search_common.cuh"

namespace prnu {

// ---------------------------------------------------------------- kernels

// Warp (optional) + row FFT of two rows per thread group; writes the packed
// half spectrum of both rows.  grid = (ceil((H/2)/ppb), wave), block = ppb*T.
// Without WARP the input is the single image at a.resid (minus *mean_sub).
template <int DT, bool WARP>
__global__ void __launch_bounds__(512) k_row_forward(PassArgs a, const float* __restrict__ mean_sub,
                                                      float2* __restrict__ out_override) {
  extern __shared__ float2 smem[];
  const int T = a.row_threads;
  const int grp = threadIdx.x / T, t = threadIdx.x - grp * T;
  const int H = a.H, W = a.W, Wh = W >> 1;
  const int pair = blockIdx.x * a.pairs_per_block + grp;
  const bool active = pair < (H >> 1);
  const int slot = blockIdx.y;
  float2* buf = smem + (size_t)grp * 2 * row_smem_len(W);
  float2* buf2 = buf + row_smem_len(W);
  const int y0 = 2 * pair, y1 = y0 + 1;
  if (active) {
    if constexpr (WARP) {
      const WorkItem it = item_of(a, slot);
      size_t base;
      const void* Rf = frame_of(a, it.frame, &base);
      const float cx = 0.5f * (float)(W - 1), cy = 0.5f * (float)(H - 1);
      const float dy0 = (float)y0 - cy, dy1 = (float)y1 - cy;
      const float bx0 = fmaf(it.a12, dy0, cx), by0 = fmaf(it.a22, dy0, cy);
      const float bx1 = fmaf(it.a12, dy1, cx), by1 = fmaf(it.a22, dy1, cy);
      for (int x = t; x < W; x += T) {
        const float dx = (float)x - cx;
        const float v0 = bilinear<DT>(Rf, base, H, W, a.rpitch, fmaf(it.a11, dx, bx0), fmaf(it.a21, dx, by0));
        const float v1 = bilinear<DT>(Rf, base, H, W, a.rpitch, fmaf(it.a11, dx, bx1), fmaf(it.a21, dx, by1));
        buf[rpad(x)] = make_float2(v0, v1);
      }
    } else {
      const float m = mean_sub ? *mean_sub : 0.f;
      for (int x = t; x < W; x += T) {
        const float v0 = load_store_type<DT>(a.resid, (size_t)y0 * W + x) - m;
        const float v1 = load_store_type<DT>(a.resid, (size_t)y1 * W + x) - m;
        buf[rpad(x)] = make_float2(v0, v1);
      }
    }
  }
  __syncthreads();
  buf = fft_row<false>(buf, buf2, a.prow, a.tw, active ? t : (1 << 28), T);
  if (active) {
    float2* o0 = (out_override ? out_override : a.spec + (size_t)slot * H * Wh) + (size_t)y0 * Wh;
    float2* o1 = o0 + Wh;
    for (int k = t; k < Wh; k += T) {
      float2 A, B;
      if (k == 0) {
        const float2 z0 = buf[rpad(0)], zn = buf[rpad(Wh)];
        A = make_float2(z0.x, zn.x);
        B = make_float2(z0.y, zn.y);
      } else {
        const float2 zk = buf[rpad(k)], zm = buf[rpad(W - k)];
        A = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        B = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
      }
      o0[k] = A;
      o1[k] = B;
    }
  }
}

// Column pass over a strip of 1 << col_log2 columns of one candidate's packed
// spectrum.  grid = (ceil((W/2) >> lg), wave), block = T.
// mode 0: fwd FFT, x conj(.) * K0^, inv FFT;  1: fwd FFT to out (fingerprint);
// 2: product only;  3: fwd FFT only;  4: inv FFT only (modes 2-4 in place).
__global__ void __launch_bounds__(512) k_col(PassArgs a, int mode, float2* __restrict__ out_f32,
                                              __half2* __restrict__ out_f16, const float* __restrict__ out_scale) {
  extern __shared__ float2 smem[];
  const int T = blockDim.x, tid = threadIdx.x;
  const int H = a.H, Wh = a.W >> 1;
  const int lg = a.col_log2, NC = 1 << lg;
  const int c0 = blockIdx.x << lg;
  const int slot = blockIdx.y;
  float2* Z = a.spec + (size_t)slot * H * Wh;
  const int n = H << lg;
  float2* buf = smem;
  float2* buf2 = smem + n;
  for (int e = tid; e < n; e += T) {
    const int i = e >> lg, col = c0 + (e & (NC - 1));
    buf[e] = col < Wh ? Z[(size_t)i * Wh + col] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  if (mode == 0 || mode == 1 || mode == 3) {
    float2* r = fft_col<false>(buf, buf2, a.pcol, a.tw, tid, T, lg);
    if (r != buf) { buf2 = buf; buf = r; }
  }
  if (mode == 1) {
    const float s = out_scale ? *out_scale : 1.f;
    for (int e = tid; e < n; e += T) {
      const int i = e >> lg, col = c0 + (e & (NC - 1));
      if (col >= Wh) continue;
      const float2 v = make_float2(buf[e].x * s, buf[e].y * s);
      if (out_f16) out_f16[(size_t)i * Wh + col] = __float22half2_rn(v);
      else out_f32[(size_t)i * Wh + col] = v;
    }
    return;
  }
  if (mode == 0 || mode == 2) {
    const WorkItem it = item_of(a, slot);
    const FpDesc fp = a.fps[it.fp];
    for (int e = tid; e < n; e += T) {
      const int i = e >> lg, col = c0 + (e & (NC - 1));
      if (col == 0 || col >= Wh) continue;
      const float2 s = load_spec(fp.spec, fp.dtype, (size_t)i * Wh + col);
      buf[e] = c_conj_mul(buf[e], s);
    }
    if (c0 == 0) {
      // packed column 0 = DC column + i * Nyquist column of both spectra:
      // separate, take conj(X^) K0^ of each, recombine.
      for (int i = tid; i <= (H >> 1); i += T) {
        const int im = (H - i) % H;
        const float2 F = buf[i << lg], Fm = buf[im << lg];
        const float2 S = load_spec(fp.spec, fp.dtype, (size_t)i * Wh);
        const float2 Sm = load_spec(fp.spec, fp.dtype, (size_t)im * Wh);
        const float2 A = make_float2(0.5f * (F.x + Fm.x), 0.5f * (F.y - Fm.y));
        const float2 B = make_float2(0.5f * (F.y + Fm.y), 0.5f * (Fm.x - F.x));
        const float2 Ka = make_float2(0.5f * (S.x + Sm.x), 0.5f * (S.y - Sm.y));
        const float2 Kb = make_float2(0.5f * (S.y + Sm.y), 0.5f * (Sm.x - S.x));
        const float2 p1 = c_conj_mul(A, Ka), p2 = c_conj_mul(B, Kb);
        const float2 q1 = c_mulc(A, Ka), q2 = c_mulc(B, Kb);
        buf[i << lg] = make_float2(p1.x - p2.y, p1.y + p2.x);
        buf[im << lg] = make_float2(q1.x - q2.y, q1.y + q2.x);
      }
    }
    __syncthreads();
  }
  if (mode == 0 || mode == 4) buf = fft_col<true>(buf, buf2, a.pcol, a.tw, tid, T, lg);
  for (int e = tid; e < n; e += T) {
    const int i = e >> lg, col = c0 + (e & (NC - 1));
    if (col < Wh) Z[(size_t)i * Wh + col] = buf[e];
  }
}

// Inverse row FFT of two rows per group; per-row max / first arg-max / sum of
// squares into a.stats, or (c_out != nullptr) the rows of C themselves.
__global__ void __launch_bounds__(512) k_row_inverse(PassArgs a, float* __restrict__ c_out) {
  extern __shared__ float2 smem[];
  const int T = a.row_threads;
  const int grp = threadIdx.x / T, t = threadIdx.x - grp * T;
  const int H = a.H, W = a.W, Wh = W >> 1;
  const int ppb = a.pairs_per_block;
  const int pair = blockIdx.x * ppb + grp;
  const bool active = pair < (H >> 1);
  const int slot = blockIdx.y;
  float2* buf = smem + (size_t)grp * 2 * row_smem_len(W);
  float2* buf2 = buf + row_smem_len(W);
  WarpRed* red = reinterpret_cast<WarpRed*>(smem + (size_t)ppb * 2 * row_smem_len(W)) + grp * 32;
  const float2* Z = a.spec + (size_t)slot * H * Wh;
  if (active) build_full_row(buf, Z + (size_t)(2 * pair) * Wh, Z + (size_t)(2 * pair + 1) * Wh, W, t, T);
  __syncthreads();
  buf = fft_row<true>(buf, buf2, a.prow, a.tw, active ? t : (1 << 28), T);
  if (c_out) {
    if (active) {
      float* ra = c_out + (size_t)(2 * pair) * W;
      for (int x = t; x < W; x += T) {
        const float2 v = buf[rpad(x)];
        ra[x] = v.x;
        ra[W + x] = v.y;
      }
    }
    return;
  }
  float ma = -INFINITY, mb = -INFINITY;
  int ia = INT_MAX, ib = INT_MAX;
  float sa = 0.f, sb = 0.f;
  if (active) {
    for (int x = t; x < W; x += T) {
      const float2 v = buf[rpad(x)];
      if (v.x > ma) { ma = v.x; ia = x; }
      if (v.y > mb) { mb = v.y; ib = x; }
      sa = fmaf(v.x, v.x, sa);
      sb = fmaf(v.y, v.y, sb);
    }
  }
  row_stats_warp(ma, ia, mb, ib, sa, sb, t, reinterpret_cast<RowRed*>(red));
  __syncthreads();
  if (active && t == 0) row_stats_final(reinterpret_cast<const RowRed*>(red), T >> 5, a.stats + (size_t)slot * H + 2 * pair);
}

// One block per candidate of the wave: see finalize_body.
__global__ void __launch_bounds__(512) k_finalize(PassArgs a) {
  extern __shared__ float2 smem[];
  finalize_body(a, blockIdx.x, blockIdx.x, smem);
}

// Best candidate of each (frame, fingerprint) group g: its items are
// first + k*share (k < count) with first = gstart[g / share] + g % share and
// count = (gstart[g / share + 1] - gstart[g / share]) / share, in ascending
// candidate order (share = 1: contiguous groups).  One warp per group.
__global__ void k_argmax(const CandResult* __restrict__ res, const WorkItem* __restrict__ items,
                         const int* __restrict__ gstart, int ngroups, int share, prnu_result* __restrict__ out,
                         int H, int W) {
  const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (g >= ngroups) return;
  argmax_group(res, items, gstart, share, out, H, W, g, threadIdx.x & 31);
}

__global__ void k_scatter_all(const CandResult* __restrict__ res, int n, int cmax, double* __restrict__ all) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) all[(size_t)res[k].group * cmax + res[k].cand] = res[k].pce;
}

// sum and sum of squares of K, double partials per block
__global__ void k_fp_partials(const float* __restrict__ K, size_t n, double* __restrict__ partials) {
  __shared__ double s1[32], s2[32];
  double a = 0, b = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = K[i];
    a += v;
    b += v * v;
  }
  a = warp_sum(a);
  b = warp_sum(b);
  if ((threadIdx.x & 31) == 0) { s1[threadIdx.x >> 5] = a; s2[threadIdx.x >> 5] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) { a += s1[k]; b += s2[k]; }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

__global__ void k_fp_finish(const double* __restrict__ partials, int nblk, size_t n, int half,
                            float* mean_out, float* scale_out, float* inv_scale_out) {
  if (threadIdx.x != 0) return;
  double a = 0, b = 0;
  for (int k = 0; k < nblk; ++k) { a += partials[2 * k]; b += partials[2 * k + 1]; }
  const double mean = a / (double)n;
  double ss = b - (double)n * mean * mean;          // sum of (K - mean)^2
  if (ss < 0) ss = 0;
  double s = 1.0;
  // FP16 storage: scale the spectrum to unit RMS magnitude (Parseval:
  // mean |K0^|^2 = sum K0^2 for the unnormalised DFT).
  if (half && ss > 0) s = 1.0 / sqrt(ss);
  *mean_out = (float)mean;
  *scale_out = (float)s;
  *inv_scale_out = (float)(1.0 / (double)(float)s);
}

// ---------------------------------------------------------------- naive per-candidate path

__global__ void k_naive_warp(PassArgs a, float* __restrict__ X) {
  const WorkItem it = a.items[a.item0];
  const int H = a.H, W = a.W;
  const size_t base = (size_t)it.frame * H * W;
  const float cx = 0.5f * (float)(W - 1), cy = 0.5f * (float)(H - 1);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)H * W;
       i += (size_t)gridDim.x * blockDim.x) {
    const int y = (int)(i / W), x = (int)(i - (size_t)y * W);
    const float dx = (float)x - cx, dy = (float)y - cy;
    const float qx = fmaf(it.a11, dx, fmaf(it.a12, dy, cx));
    const float qy = fmaf(it.a21, dx, fmaf(it.a22, dy, cy));
    X[i] = bilinear<kF32>(a.resid, base, H, W, W, qx, qy);
  }
}

__global__ void k_naive_reduce(const float* __restrict__ C, size_t n, float* bmax, int* barg, double* bsum) {
  __shared__ float sm[32];
  __shared__ int si[32];
  __shared__ double ss[32];
  float v = -INFINITY;
  int vi = INT_MAX;
  double s = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float c = C[i];
    better_f(v, vi, c, (int)i);
    s += (double)c * c;
  }
  warp_maxarg(v, vi);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) { sm[threadIdx.x >> 5] = v; si[threadIdx.x >> 5] = vi; ss[threadIdx.x >> 5] = s; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) { better_f(v, vi, sm[k], si[k]); s += ss[k]; }
    bmax[blockIdx.x] = v;
    barg[blockIdx.x] = vi;
    bsum[blockIdx.x] = s;
  }
}

__global__ void k_naive_final(const float* __restrict__ C, int H, int W, const WorkItem* __restrict__ itp,
                              const FpDesc* __restrict__ fps, const float* __restrict__ scale,
                              const float* bmax, const int* barg, const double* bsum, int nblk,
                              CandResult* __restrict__ out) {
  if (threadIdx.x != 0) return;
  float v = -INFINITY;
  int vi = INT_MAX;
  double tot = 0;
  for (int k = 0; k < nblk; ++k) { better_f(v, vi, bmax[k], barg[k]); tot += bsum[k]; }
  if (vi == INT_MAX) vi = 0;
  const int py = vi / W, px = vi - py * W;
  double win = 0;
  for (int dy = -kHalfWindow; dy <= kHalfWindow; ++dy)
    for (int dx = -kHalfWindow; dx <= kHalfWindow; ++dx) {
      const double c = C[(size_t)((py + dy + H) % H) * W + (px + dx + W) % W];
      win += c * c;
    }
  double E = (tot - win) / ((double)H * W - kWindowCount);
  if (E < 0) E = 0;
  const double pk = v;
  double pce;
  if (E > 0.0) pce = (pk < 0 ? -1.0 : 1.0) * pk * pk / E;
  else pce = pk == 0.0 ? 0.0 : (pk < 0 ? -INFINITY : INFINITY);
  const WorkItem it = *itp;
  double pv = pk / ((double)H * W) * (double)(*fps[it.fp].inv_scale);
  if (scale) pv /= (double)scale[it.frame];
  CandResult r;
  r.pce = pce;
  r.peak = (float)pv;
  r.py = py;
  r.px = px;
  r.cand = it.cand;
  r.group = it.group;
  r.pad = 0;
  *out = r;
}

// ---------------------------------------------------------------- launchers

#define PRNU_LAUNCH_CHECK()                                                                 \
  do {                                                                                      \
    cudaError_t e_ = cudaGetLastError();                                                    \
    if (e_ != cudaSuccess) throw Error{PRNU_ECUDA, std::string(__func__) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

void launch_row_forward(const PassArgs& a, bool warp, const float* mean_sub, float2* out, cudaStream_t s,
                        LaunchCounter& lc) {
  int T, maxb;
  row_launch_shape(a.prow, &T, &maxb);
  PRNU_CHECK_ARG(T == a.row_threads, "row thread count mismatch");
  const int ppb = a.pairs_per_block;
  dim3 g((a.H / 2 + ppb - 1) / ppb, a.nitems), b(ppb * T);
  const size_t sm = row_smem_bytes(a.W, ppb);
  ProfScope ps(lc, kKindRowForward, s);
  if (warp) {
    if (a.rdtype == kF32) k_row_forward<kF32, true><<<g, b, sm, s>>>(a, mean_sub, out);
    else if (a.rdtype == kF16) k_row_forward<kF16, true><<<g, b, sm, s>>>(a, mean_sub, out);
    else k_row_forward<kBF16, true><<<g, b, sm, s>>>(a, mean_sub, out);
  } else {
    if (a.rdtype == kF32) k_row_forward<kF32, false><<<g, b, sm, s>>>(a, mean_sub, out);
    else if (a.rdtype == kF16) k_row_forward<kF16, false><<<g, b, sm, s>>>(a, mean_sub, out);
    else k_row_forward<kBF16, false><<<g, b, sm, s>>>(a, mean_sub, out);
  }
  PRNU_LAUNCH_CHECK();
  lc.n++;
}

void launch_col(const PassArgs& a, int mode, float2* out_f32, void* out_f16, const float* scale, cudaStream_t s,
                LaunchCounter& lc) {
  int T, maxb;
  col_launch_shape(a.pcol, a.col_log2, &T, &maxb);
  const int Wh = a.W / 2;
  const int nc = 1 << a.col_log2;
  dim3 g((Wh + nc - 1) / nc, a.nitems), b(T);
  const size_t sm = 2 * (size_t)a.H * nc * sizeof(float2);
  __half2* o16 = reinterpret_cast<__half2*>(out_f16);
  ProfScope ps(lc, kKindColumn, s);
  k_col<<<g, b, sm, s>>>(a, mode, out_f32, o16, scale);
  PRNU_LAUNCH_CHECK();
  lc.n++;
}

void launch_row_inverse(const PassArgs& a, float* c_out, cudaStream_t s, LaunchCounter& lc) {
  int T, maxb;
  row_launch_shape(a.prow, &T, &maxb);
  const int ppb = a.pairs_per_block;
  dim3 g((a.H / 2 + ppb - 1) / ppb, a.nitems), b(ppb * T);
  const size_t sm = row_smem_bytes(a.W, ppb);
  ProfScope ps(lc, kKindRowInverse, s);
  k_row_inverse<<<g, b, sm, s>>>(a, c_out);
  PRNU_LAUNCH_CHECK();
  lc.n++;
}

void launch_finalize(const PassArgs& a, cudaStream_t s, LaunchCounter& lc) {
  int T, maxb;
  row_launch_shape(a.prow, &T, &maxb);
  dim3 g(a.nitems), b(T);
  const size_t sm = row_smem_bytes(a.W, 1);
  ProfScope ps(lc, kKindFinalize, s);
  k_finalize<<<g, b, sm, s>>>(a);
  PRNU_LAUNCH_CHECK();
  lc.n++;
}

void launch_argmax(const CandResult* res, const WorkItem* items, const int* group_start, int ngroups, int share,
                   prnu_result* out, const float* /*scale*/, int H, int W, cudaStream_t s, LaunchCounter& lc) {
  if (ngroups <= 0) return;
  const int warps = 8;
  ProfScope ps(lc, kKindArgmax, s);
  k_argmax<<<(ngroups + warps - 1) / warps, warps * 32, 0, s>>>(res, items, group_start, ngroups,
                                                                std::max(share, 1), out, H, W);
  PRNU_LAUNCH_CHECK();
  lc.n++;
}

void launch_scatter_all(const CandResult* res, int nitems, int cmax, double* all, cudaStream_t s, LaunchCounter& lc) {
  if (nitems <= 0) return;
  ProfScope ps(lc, kKindScatter, s);
  k_scatter_all<<<(nitems + 255) / 256, 256, 0, s>>>(res, nitems, cmax, all);
  PRNU_LAUNCH_CHECK();
  lc.n++;
}

void launch_fp_stats(const float* K, int H, int W, double* partials, int nblk, float* mean_out, float* scale_out,
                     float* inv_scale_out, bool half, cudaStream_t s, LaunchCounter& lc) {
  ProfScope ps(lc, kKindFpSpectrum, s);
  k_fp_partials<<<nblk, 256, 0, s>>>(K, (size_t)H * W, partials);
  PRNU_LAUNCH_CHECK();
  k_fp_finish<<<1, 32, 0, s>>>(partials, nblk, (size_t)H * W, half ? 1 : 0, mean_out, scale_out, inv_scale_out);
  PRNU_LAUNCH_CHECK();
  lc.n += 2;
}

void launch_naive_warp(const PassArgs& a, float* X, cudaStream_t s, LaunchCounter& lc) {
  ProfScope ps(lc, kKindNaiveWarp, s);
  k_naive_warp<<<1024, 256, 0, s>>>(a, X);
  PRNU_LAUNCH_CHECK();
  lc.n++;
}

void launch_naive_pce(const float* C, int H, int W, const WorkItem* item, const FpDesc* fps, const float* scale,
                      CandResult* out, float* bmax, int* barg, double* bsum, int nblk, cudaStream_t s,
                      LaunchCounter& lc) {
  ProfScope ps(lc, kKindNaivePce, s);
  k_naive_reduce<<<nblk, 256, 0, s>>>(C, (size_t)H * W, bmax, barg, bsum);
  PRNU_LAUNCH_CHECK();
  k_naive_final<<<1, 32, 0, s>>>(C, H, W, item, fps, scale, bmax, barg, bsum, nblk, out);
  PRNU_LAUNCH_CHECK();
  lc.n += 2;
}

const char* const kKindNames[kKindCount] = {"residual", "fingerprint_spectrum", "row_forward", "column",
                                             "row_inverse", "finalize", "argmax", "scatter", "naive_warp",
                                             "naive_pce", "fused"};

cudaEvent_t LaunchCounter::take() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  PRNU_CUDA_TRY(cudaEventCreate(&e));
  return e;
}

void LaunchCounter::start(int kind, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(mu);
  Rec r{kind, take(), take()};
  PRNU_CUDA_TRY(cudaEventRecord(r.a, s));
  recs.push_back(r);
}

void LaunchCounter::stop(cudaStream_t s) {
  std::lock_guard<std::mutex> lk(mu);
  if (!recs.empty()) cudaEventRecord(recs.back().b, s);
}

template <class K>
static void allow_smem(K k) {
  allow_max_dynamic_smem(k);
}

void set_kernel_attributes() {
  allow_smem(k_row_forward<kF32, true>);
  allow_smem(k_row_forward<kF16, true>);
  allow_smem(k_row_forward<kBF16, true>);
  allow_smem(k_row_forward<kF32, false>);
  allow_smem(k_row_forward<kF16, false>);
  allow_smem(k_row_forward<kBF16, false>);
  allow_smem(k_col);
  allow_smem(k_row_inverse);
  allow_smem(k_finalize);
  cudaGetLastError();
}

}  // namespace prnu
