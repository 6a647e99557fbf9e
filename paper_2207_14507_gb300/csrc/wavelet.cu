// wavelet.cu -- noise residual by Mihcak's wavelet denoiser (the paper's
// denoiser, Sec. 2.2), as an alternative to the 3x3 Wiener residual.
//
// Per frame (FP32 throughout):
//   1. the frame, mirrored at its bottom and right edges up to multiples of
//      16 (Hp x Wp), as float;
//   2. four levels of the orthonormal separable transform with Daubechies'
//      8-tap filter, periodic: rows (low half | high half), then columns (low
//      half over high half), each level on the previous level's low-low
//      quadrant (the quadrant layout keeps every band at pitch Wp);
//   3. every detail coefficient c replaced by its noise part
//      c s0^2 / (s2 + s0^2), s2 = min over W in {3, 5, 7, 9} of
//      max(0, mean of c^2 over the W x W window of its band - s0^2), zeros
//      outside the band; the last low-low band replaced by 0;
//   4. the inverse transform of those noise parts: W(I) = I - F(I) (the
//      transform is linear), cropped to H x W; R = I W(I) or W(I).
// Two Hp x Wp buffers per frame: the coefficients (A) and a scratch (T); the
// noise parts and the inverse run in T and A alternately.
#include <algorithm>

#include "internal.h"

namespace prnu {

namespace {

// Daubechies' scaling filter with 4 vanishing moments, sum sqrt(2); wavelet
// filter g[k] = (-1)^k h[7 - k]
__constant__ float c_h[8] = {0.2303778133088964f,  0.7148465705529154f,  0.6308807679298587f,
                             -0.0279837694168599f, -0.1870348117190931f, 0.0308413818355607f,
                             0.0328830116668852f,  -0.0105974017850690f};
__device__ __forceinline__ float wav_g(int k) { return (k & 1) ? -c_h[7 - k] : c_h[7 - k]; }

constexpr int kWB = 128;

__global__ void k_wav_pad(const uint8_t* __restrict__ frames, size_t pitch, int H, int W, int Hp, int Wp,
                          float* __restrict__ A) {
  const int x = blockIdx.x * kWB + threadIdx.x, y = blockIdx.y, f = blockIdx.z;
  if (x >= Wp) return;
  const int ys = y < H ? y : 2 * H - 1 - y, xs = x < W ? x : 2 * W - 1 - x;   // half-sample mirror
  A[((size_t)f * Hp + y) * Wp + x] = (float)frames[((size_t)f * H + ys) * pitch + xs];
}

// rows of the h x w top-left region of X (pitch Wp) -> T: [low w/2 | high w/2]
__global__ void k_wav_rows(const float* __restrict__ X, int w, int Hp, int Wp, float* __restrict__ T) {
  const int n = blockIdx.x * kWB + threadIdx.x, y = blockIdx.y, f = blockIdx.z;
  const int w2 = w / 2;
  if (n >= w2) return;
  const float* row = X + ((size_t)f * Hp + y) * Wp;
  float a = 0.f, d = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float v = row[(2 * n + k) % w];
    a = fmaf(c_h[k], v, a);
    d = fmaf(wav_g(k), v, d);
  }
  float* o = T + ((size_t)f * Hp + y) * Wp;
  o[n] = a;
  o[w2 + n] = d;
}

// columns of the h x w top-left region of T -> X: low h/2 rows over high h/2 rows
__global__ void k_wav_cols(const float* __restrict__ T, int h, int w, int Hp, int Wp, float* __restrict__ X) {
  const int x = blockIdx.x * kWB + threadIdx.x, n = blockIdx.y, f = blockIdx.z;
  if (x >= w) return;
  const float* base = T + (size_t)f * Hp * Wp + x;
  float a = 0.f, d = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float v = base[(size_t)((2 * n + k) % h) * Wp];
    a = fmaf(c_h[k], v, a);
    d = fmaf(wav_g(k), v, d);
  }
  float* o = X + (size_t)f * Hp * Wp + x;
  o[(size_t)n * Wp] = a;
  o[(size_t)(h / 2 + n) * Wp] = d;
}

// inverse of k_wav_cols: X (h x w region, low over high) -> T
__global__ void k_wav_icols(const float* __restrict__ X, int h, int w, int Hp, int Wp, float* __restrict__ T) {
  const int x = blockIdx.x * kWB + threadIdx.x, m = blockIdx.y, f = blockIdx.z;
  if (x >= w) return;
  const int h2 = h / 2;
  const float* base = X + (size_t)f * Hp * Wp + x;
  float v = 0.f;
#pragma unroll
  for (int k = (m & 1); k < 8; k += 2) {   // output m takes input 2n + k = m (mod h)
    const int n = (((m - k) / 2) % h2 + h2) % h2;
    v = fmaf(c_h[k], base[(size_t)n * Wp], v);
    v = fmaf(wav_g(k), base[(size_t)(h2 + n) * Wp], v);
  }
  T[((size_t)f * Hp + m) * Wp + x] = v;
}

// inverse of k_wav_rows: T (h x w region, [low | high]) -> X
__global__ void k_wav_irows(const float* __restrict__ T, int w, int Hp, int Wp, float* __restrict__ X) {
  const int m = blockIdx.x * kWB + threadIdx.x, y = blockIdx.y, f = blockIdx.z;
  if (m >= w) return;
  const int w2 = w / 2;
  const float* row = T + ((size_t)f * Hp + y) * Wp;
  float v = 0.f;
#pragma unroll
  for (int k = (m & 1); k < 8; k += 2) {
    const int n = (((m - k) / 2) % w2 + w2) % w2;
    v = fmaf(c_h[k], row[n], v);
    v = fmaf(wav_g(k), row[w2 + n], v);
  }
  X[((size_t)f * Hp + y) * Wp + m] = v;
}

// noise parts of the three detail bands (h2 x w2 each) of one level: band b of
// frame f = blockIdx.z: 0 (rows high, columns low) at (0, w2), 1 at (h2, 0),
// 2 at (h2, w2); reads A, writes T
constexpr int kSX = 32, kSY = 8, kSR = 4;
__global__ void __launch_bounds__(kSX * kSY) k_wav_shrink(const float* __restrict__ A, int h2, int w2, int Hp, int Wp,
                                                        float s0sq, float* __restrict__ T) {
  __shared__ float sq[(kSY + 2 * kSR) * (kSX + 2 * kSR)];
  const int f = blockIdx.z / 3, b = blockIdx.z - 3 * f;
  const int oy = b == 0 ? 0 : h2, ox = b == 1 ? 0 : w2;
  const float* band = A + ((size_t)f * Hp + oy) * Wp + ox;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kSX + tx;
  const int bx0 = blockIdx.x * kSX - kSR, by0 = blockIdx.y * kSY - kSR;
  constexpr int SW = kSX + 2 * kSR, SN = (kSY + 2 * kSR) * SW;
  for (int k = tid; k < SN; k += kSX * kSY) {
    const int sy = k / SW, sx = k - sy * SW;
    const int y = by0 + sy, x = bx0 + sx;
    float v = 0.f;
    if (y >= 0 && y < h2 && x >= 0 && x < w2) {
      const float c = band[(size_t)y * Wp + x];
      v = c * c;
    }
    sq[k] = v;
  }
  __syncthreads();
  const int x = blockIdx.x * kSX + tx, y = blockIdx.y * kSY + ty;
  if (x >= w2 || y >= h2) return;
  // window sums of radius 1..4 around (ty, tx) + kSR, ring by ring
  float sum = 0.f, s2 = INFINITY;
  const float* cen = sq + (ty + kSR) * SW + tx + kSR;
  sum = cen[0];
#pragma unroll
  for (int r = 1; r <= kSR; ++r) {
#pragma unroll
    for (int d = -r; d <= r; ++d) {
      sum += cen[-r * SW + d] + cen[r * SW + d];
      if (d > -r && d < r) sum += cen[d * SW - r] + cen[d * SW + r];
    }
    const float nw = (float)((2 * r + 1) * (2 * r + 1));
    s2 = fminf(s2, fmaxf(sum / nw - s0sq, 0.f));
  }
  const float c = band[(size_t)y * Wp + x];
  const float den = s2 + s0sq;
  T[((size_t)f * Hp + oy + y) * Wp + ox + x] = den > 0.f ? c * s0sq / den : 0.f;
}

__global__ void k_wav_zero(int h, int w, int Hp, int Wp, float* __restrict__ T) {
  const int x = blockIdx.x * kWB + threadIdx.x, y = blockIdx.y, f = blockIdx.z;
  if (x < w) T[((size_t)f * Hp + y) * Wp + x] = 0.f;
}

// R = I W (or W) of frame f0 + blockIdx.z into out (dense [F][H][W] of type DT).
// MODE 0: store R; MODE 1: per-block sum of R^2 to partials; MODE 2: store R * scale[f].
template <int DT, int MODE>
__global__ void k_wav_out(const float* __restrict__ Wr, const uint8_t* __restrict__ frames, size_t pitch, int H, int W,
                          int Hp, int Wp, int f0, int weight, void* __restrict__ out, double* __restrict__ partials,
                          const float* __restrict__ scale) {
  __shared__ double part[kWB / 32];
  const int x = blockIdx.x * kWB + threadIdx.x, y = blockIdx.y, fl = blockIdx.z, f = f0 + fl;
  float r = 0.f;
  if (x < W) {
    const float w = Wr[((size_t)fl * Hp + y) * Wp + x];
    r = weight ? (float)frames[((size_t)f * H + y) * pitch + x] * w : w;
    const size_t o = ((size_t)f * H + y) * W + x;
    if (MODE == 0) store_store_type<DT>(out, o, r);
    if (MODE == 2) store_store_type<DT>(out, o, r * scale[f]);
  }
  if (MODE == 1) {   // float within a warp, double across warps and blocks
    float v = r * r;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = (double)v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int k = 0; k < kWB / 32; ++k) s += part[k];
      partials[(size_t)f * gridDim.x * gridDim.y + (size_t)y * gridDim.x + blockIdx.x] = s;
    }
  }
}

template <int MODE>
void wav_out(int dtype, dim3 g, cudaStream_t s, const float* Wr, const uint8_t* frames, size_t pitch, int H, int W,
             int Hp, int Wp, int f0, int weight, void* out, double* partials, const float* scale) {
  if (dtype == kF32)
    k_wav_out<kF32, MODE><<<g, kWB, 0, s>>>(Wr, frames, pitch, H, W, Hp, Wp, f0, weight, out, partials, scale);
  else if (dtype == kF16)
    k_wav_out<kF16, MODE><<<g, kWB, 0, s>>>(Wr, frames, pitch, H, W, Hp, Wp, f0, weight, out, partials, scale);
  else
    k_wav_out<kBF16, MODE><<<g, kWB, 0, s>>>(Wr, frames, pitch, H, W, Hp, Wp, f0, weight, out, partials, scale);
  PRNU_CUDA_TRY(cudaGetLastError());
}

}  // namespace

size_t wavelet_partials_needed(int F, int H, int W) { return (size_t)F * H * ((W + kWB - 1) / kWB); }

namespace {

// W(I) of nf frames into bufT (pitch Wp, frame stride Hp*Wp); bufA is scratch
void wavelet_chunk(const uint8_t* fr, int nf, int H, int W, size_t pitch, float s0sq, float* bufA, float* bufT,
                   cudaStream_t s, LaunchCounter& lc) {
  constexpr int kLevels = 4;
  const int Hp = (H + 15) / 16 * 16, Wp = (W + 15) / 16 * 16;
  k_wav_pad<<<dim3((Wp + kWB - 1) / kWB, Hp, nf), kWB, 0, s>>>(fr, pitch, H, W, Hp, Wp, bufA);
  PRNU_CUDA_TRY(cudaGetLastError());
  lc.n++;
  for (int l = 0; l < kLevels; ++l) {   // forward: A -> T (rows) -> A (columns)
    const int h = Hp >> l, w = Wp >> l;
    k_wav_rows<<<dim3((w / 2 + kWB - 1) / kWB, h, nf), kWB, 0, s>>>(bufA, w, Hp, Wp, bufT);
    k_wav_cols<<<dim3((w + kWB - 1) / kWB, h / 2, nf), kWB, 0, s>>>(bufT, h, w, Hp, Wp, bufA);
    PRNU_CUDA_TRY(cudaGetLastError());
    lc.n += 2;
  }
  for (int l = 0; l < kLevels; ++l) {   // noise parts of the detail bands: A -> T
    const int h2 = (Hp >> l) / 2, w2 = (Wp >> l) / 2;
    k_wav_shrink<<<dim3((w2 + kSX - 1) / kSX, (h2 + kSY - 1) / kSY, 3 * nf), dim3(kSX, kSY), 0, s>>>(
        bufA, h2, w2, Hp, Wp, s0sq, bufT);
    PRNU_CUDA_TRY(cudaGetLastError());
    lc.n++;
  }
  {
    const int h = Hp >> kLevels, w = Wp >> kLevels;
    k_wav_zero<<<dim3((w + kWB - 1) / kWB, h, nf), kWB, 0, s>>>(h, w, Hp, Wp, bufT);
    PRNU_CUDA_TRY(cudaGetLastError());
    lc.n++;
  }
  for (int l = kLevels - 1; l >= 0; --l) {   // inverse: T (columns) -> A (rows) -> T
    const int h = Hp >> l, w = Wp >> l;
    k_wav_icols<<<dim3((w + kWB - 1) / kWB, h, nf), kWB, 0, s>>>(bufT, h, w, Hp, Wp, bufA);
    k_wav_irows<<<dim3((w + kWB - 1) / kWB, h, nf), kWB, 0, s>>>(bufA, w, Hp, Wp, bufT);
    PRNU_CUDA_TRY(cudaGetLastError());
    lc.n += 2;
  }
}

}  // namespace

void launch_wavelet_residual(const uint8_t* frames, int F, int H, int W, size_t pitch, int flags, int dtype,
                             float sigma0, void* out, float* scale, float* bufA, float* bufT, int chunk,
                             double* partials, cudaStream_t s, LaunchCounter& lc) {
  const int Hp = (H + 15) / 16 * 16, Wp = (W + 15) / 16 * 16;
  const int weight = (flags & PRNU_WEIGHT_BY_INTENSITY) ? 1 : 0;
  const bool norm = (flags & PRNU_NORMALISE) != 0;
  const float s0sq = sigma0 * sigma0;
  const int gx = (W + kWB - 1) / kWB;
  ProfScope ps(lc, kKindResidual, s);
  for (int f0 = 0; f0 < F; f0 += chunk) {
    const int nf = std::min(chunk, F - f0);
    wavelet_chunk(frames + (size_t)f0 * H * pitch, nf, H, W, pitch, s0sq, bufA, bufT, s, lc);
    if (norm) wav_out<1>(dtype, dim3(gx, H, nf), s, bufT, frames, pitch, H, W, Hp, Wp, f0, weight, out, partials, scale);
    else wav_out<0>(dtype, dim3(gx, H, nf), s, bufT, frames, pitch, H, W, Hp, Wp, f0, weight, out, partials, scale);
    lc.n++;
  }
  if (norm) {   // s = 1 / RMS(R) per frame, then the scaled store
    launch_resid_scale(partials, gx * H, F, H, W, scale, s, lc);
    for (int f0 = 0; f0 < F; f0 += chunk) {
      const int nf = std::min(chunk, F - f0);
      if (F > chunk)   // the buffers hold the last chunk only: recompute
        wavelet_chunk(frames + (size_t)f0 * H * pitch, nf, H, W, pitch, s0sq, bufA, bufT, s, lc);
      wav_out<2>(dtype, dim3(gx, H, nf), s, bufT, frames, pitch, H, W, Hp, Wp, f0, weight, out, partials, scale);
      lc.n++;
    }
  } else if (scale) {
    launch_fill(scale, F, 1.f, s, lc);
  }
}

}  // namespace prnu
