// residual.cu -- noise residual of uint8 frames (Sec. 2.2, W(I) = I - F(I)),
// F = 3x3 local Wiener filter with the frame's mean local variance as the
// noise power, borders replicated.
//
// The 3x3 moments of uint8 pixels are integers: S1 = sum x, S2 = sum x^2,
// V = 9 S2 - S1^2 = 81 * (population variance), D = 9 x - S1 = 9 (x - mu).
// The frame noise power nu2 = sum V / (81 H W) is accumulated exactly in
// 64-bit integers, so it does not depend on the reduction order.  Then
//   W = (x - mu) nu2 / var = 9 D nu2 / V   where var >= nu2 (and V > 0),
//   W = x - mu = D / 9                      elsewhere,
// and R = x W (PRNU_WEIGHT_BY_INTENSITY) or W.
#include "internal.h"

namespace prnu {

namespace {

// A block covers a 32 x 32 tile with 32 x 8 threads (4 rows each); the tile
// and its one-pixel halo (borders replicated) are staged once in shared memory.
constexpr int kBX = 32, kBY = 32, kBR = 4, kTW = kBX + 2, kTH = kBY + 2;
static_assert(kBY == 8 * kBR, "a thread covers kBR rows of the tile");

__device__ __forceinline__ void load_tile_u8(const uint8_t* __restrict__ f, size_t pitch, int H, int W, int* tile) {
  const int tid = threadIdx.y * kBX + threadIdx.x;
  const int x0 = blockIdx.x * kBX - 1, y0 = blockIdx.y * kBY - 1;
  for (int k = tid; k < kTW * kTH; k += kBX * 8) {
    const int sy = k / kTW, sx = k - sy * kTW;
    const int y = min(max(y0 + sy, 0), H - 1), x = min(max(x0 + sx, 0), W - 1);
    tile[k] = __ldg(f + (size_t)y * pitch + x);
  }
  __syncthreads();
}

// 3x3 sums of x and x^2 and the centre of tile pixel (tx, ty)
__device__ __forceinline__ void moments3x3(const int* tile, int tx, int ty, int* s1, int* s2, int* xc) {
  int a = 0, b = 0;
#pragma unroll
  for (int dy = 0; dy < 3; ++dy)
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) {
      const int v = tile[(ty + dy) * kTW + tx + dx];
      a += v;
      b += v * v;
    }
  *s1 = a;
  *s2 = b;
  *xc = tile[(ty + 1) * kTW + tx + 1];
}

// per block: the integer sum of 81 * (local variance) of its pixels, one slot per block
__global__ void __launch_bounds__(kBX * 8) k_resid_moments(const uint8_t* __restrict__ frames, size_t pitch, int H,
                                                           int W, unsigned long long* __restrict__ part_out) {
  __shared__ int tile[kTW * kTH];
  __shared__ unsigned long long part[8];
  const int f = blockIdx.z;
  load_tile_u8(frames + (size_t)f * H * pitch, pitch, H, W, tile);
  const int tx = threadIdx.x, x = blockIdx.x * kBX + tx;
  unsigned long long v = 0;
#pragma unroll
  for (int k = 0; k < kBR; ++k) {
    const int ty = threadIdx.y + 8 * k, y = blockIdx.y * kBY + ty;
    if (x < W && y < H) {
      int s1, s2, xc;
      moments3x3(tile, tx, ty, &s1, &s2, &xc);
      v += (unsigned long long)(9 * s2 - s1 * s1);
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (tx == 0) part[threadIdx.y] = v;
  __syncthreads();
  if (threadIdx.y == 0 && tx == 0) {
    unsigned long long s = 0;
    for (int k = 0; k < 8; ++k) s += part[k];
    part_out[(size_t)f * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// one block per frame: acc[f] = sum of the frame's block slots (integers: exact in any order)
__global__ void k_resid_noise(const unsigned long long* __restrict__ part, int nblk,
                              unsigned long long* __restrict__ acc) {
  __shared__ unsigned long long red[32];
  const int f = blockIdx.x;
  unsigned long long v = 0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) v += part[(size_t)f * nblk + k];
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    acc[f] = t;
  }
}

__device__ __forceinline__ float residual_value(int s1, int s2, int xc, float nu2, float nu2x81, int weight) {
  const int V = 9 * s2 - s1 * s1;
  const float D = (float)(9 * xc - s1);
  float w;
  if (V > 0 && (float)V >= nu2x81) w = (9.f * D) * nu2 / (float)V;
  else w = D / 9.f;
  return weight ? (float)xc * w : w;
}

// MODE 0: store R; MODE 1: per-block sum of R^2 (double) to partials; MODE 2: store R * scale[f].
// R(y, x) of frame f goes to out[f * lay.fpitch + lay.roff + y * lay.rpitch + x].
template <int DT, int MODE>
__global__ void __launch_bounds__(kBX * 8) k_resid_apply(const uint8_t* __restrict__ frames, size_t pitch, int H,
                                                         int W, const unsigned long long* __restrict__ acc,
                                                         int weight, void* __restrict__ out,
                                                         double* __restrict__ partials,
                                                         const float* __restrict__ scale, ResidLayout lay) {
  __shared__ int tile[kTW * kTH];
  __shared__ double part[8];
  __shared__ float s_nu2[2];
  const int f = blockIdx.z;
  if (threadIdx.x == 0 && threadIdx.y == 0) {   // once per block: the FP64 pipe is narrow
    const double nu2d = (double)acc[f] / (81.0 * (double)H * (double)W);
    s_nu2[0] = (float)nu2d;
    s_nu2[1] = (float)(81.0 * nu2d);
  }
  load_tile_u8(frames + (size_t)f * H * pitch, pitch, H, W, tile);   // (synchronises)
  const float nu2 = s_nu2[0];
  const float nu2x81 = s_nu2[1];
  const int tx = threadIdx.x, x = blockIdx.x * kBX + tx;
  float sq = 0.f;
#pragma unroll
  for (int k = 0; k < kBR; ++k) {
    const int ty = threadIdx.y + 8 * k, y = blockIdx.y * kBY + ty;
    if (x < W && y < H) {
      int s1, s2, xc;
      moments3x3(tile, tx, ty, &s1, &s2, &xc);
      const float r = residual_value(s1, s2, xc, nu2, nu2x81, weight);
      const size_t o = (size_t)f * lay.fpitch + lay.roff + (size_t)y * lay.rpitch + x;
      if (MODE == 0) store_store_type<DT>(out, o, r);
      if (MODE == 2) store_store_type<DT>(out, o, r * scale[f]);
      sq = fmaf(r, r, sq);
    }
  }
  if (MODE == 1) {   // float within a warp, double across warps and blocks
    float v = sq;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (tx == 0) part[threadIdx.y] = (double)v;
    __syncthreads();
    if (threadIdx.y == 0 && tx == 0) {
      double t = 0;
      for (int k = 0; k < 8; ++k) t += part[k];
      partials[(size_t)f * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
  }
}

// one block per frame: fixed-order sum of the block partials, s = 1/RMS
__global__ void k_resid_scale(const double* __restrict__ partials, int nblk, int H, int W, float* __restrict__ scale) {
  __shared__ double part[32];
  const int f = blockIdx.x;
  double s = 0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) s += partials[(size_t)f * nblk + k];
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += part[k];
    const double ms = t / ((double)H * (double)W);
    scale[f] = ms > 0 ? (float)(1.0 / sqrt(ms)) : 1.f;
  }
}

__global__ void k_fill(float* __restrict__ p, int n, float v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// Copy of dense [F][H][W] frames into the zero-bordered layout: padded row
// yp, column xp of frame f holds pixel (yp - 1, xp - 1), or 0 outside.
template <typename T>
__global__ void k_pad_frames(const T* __restrict__ in, int H, int W, T* __restrict__ out) {
  const int P = W + 3;
  const int xp = blockIdx.x * blockDim.x + threadIdx.x, yp = blockIdx.y;
  const int f = blockIdx.z;
  if (xp >= P) return;
  const int x = xp - 1, y = yp - 1;
  T v{};
  if ((unsigned)x < (unsigned)W && (unsigned)y < (unsigned)H) v = in[((size_t)f * H + y) * W + x];
  out[(size_t)f * (H + 3) * P + (size_t)yp * P + xp] = v;
}

// The same layout for half storage as pairs: element (yp, xp) holds the
// 16-bit values of padded pixels (yp, xp) and (yp, xp + 1) (0 beyond the
// padded row), the first in the low half (the .x of a __half2).
__global__ void k_pad_pairs(const uint16_t* __restrict__ in, int H, int W, uint32_t* __restrict__ out) {
  const int P = W + 3;
  const int xp = blockIdx.x * blockDim.x + threadIdx.x, yp = blockIdx.y;
  const int f = blockIdx.z;
  if (xp >= P) return;
  const int x = xp - 1, y = yp - 1;
  uint32_t lo = 0, hi = 0;
  if ((unsigned)y < (unsigned)H) {
    const uint16_t* row = in + ((size_t)f * H + y) * W;
    if ((unsigned)x < (unsigned)W) lo = row[x];
    if ((unsigned)(x + 1) < (unsigned)W) hi = row[x + 1];
  }
  out[(size_t)f * (H + 3) * P + (size_t)yp * P + xp] = lo | (hi << 16);
}

template <int MODE>
void apply_dispatch(int dtype, dim3 g, dim3 b, cudaStream_t s, const uint8_t* frames, size_t pitch, int H, int W,
                    const unsigned long long* acc, int weight, void* out, double* partials, const float* scale,
                    const ResidLayout& l) {
  if (dtype == kF32)
    k_resid_apply<kF32, MODE><<<g, b, 0, s>>>(frames, pitch, H, W, acc, weight, out, partials, scale, l);
  else if (dtype == kF16)
    k_resid_apply<kF16, MODE><<<g, b, 0, s>>>(frames, pitch, H, W, acc, weight, out, partials, scale, l);
  else
    k_resid_apply<kBF16, MODE><<<g, b, 0, s>>>(frames, pitch, H, W, acc, weight, out, partials, scale, l);
}

// Eq. 2 sums over a chunk of Lc frames: num += sum_l R_l (R = I W(I)),
// den += sum_l I_l^2, in double (first: start from zero).
__global__ void k_fp_accumulate(const float* __restrict__ R, const uint8_t* __restrict__ frames, size_t pitch, int Lc,
                                int H, int W, double* __restrict__ num, double* __restrict__ den, int first) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W) return;
  const size_t p = (size_t)y * W + x;
  double a = first ? 0.0 : num[p], b = first ? 0.0 : den[p];
  for (int l = 0; l < Lc; ++l) {
    a += (double)R[(size_t)l * H * W + p];
    const double I = (double)frames[((size_t)l * H + y) * pitch + x];
    b += I * I;
  }
  num[p] = a;
  den[p] = b;
}

__global__ void k_fp_divide(const double* __restrict__ num, const double* __restrict__ den, float* __restrict__ K,
                            size_t n) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) K[i] = den[i] > 0.0 ? (float)(num[i] / den[i]) : 0.f;
}


// ---------------------------------------------------------------- frame-literal residuals (Sec. 3.2)
//
// The paper warps the frame for every candidate and extracts the residual of
// the warped frame.  For render r (source frame f, similarity a11..a22):
//   X(p)  = bilinear(I_f, c + A (p - c)), each tap outside the frame 0,
//   W(X)  = X - Wiener3x3(X), 3x3 moments with replicated borders, noise power
//           nu2 = mean over the frame of the local variances of X,
//   R     = X W(X) (PRNU_WEIGHT_BY_INTENSITY) or W(X).
// X is not an integer image, so the moments are taken in float from the
// differences to the window's centre (d = x_k - x_c: mean m1 = sum d / 9,
// variance sum d^2 / 9 - m1^2), which keeps the cancellation small.  A block
// warps its 32x8 tile plus a one-pixel halo into shared memory; halo pixels
// outside the frame are the warped values at the clamped position (the
// replicated border).

constexpr int kLX = 32, kLY = 32, kLR = 4, kLTX = kLX + 2, kLTY = kLY + 2;   // 32 x 8 threads, 4 rows each
static_assert(kLY == 8 * kLR, "a thread covers kLR rows of the tile");

// uint8 -> float without a conversion instruction: the byte in the low
// mantissa bits of 2^23 (exact for every byte value)
__device__ __forceinline__ float u8f(uint32_t v) { return __int_as_float(0x4B000000u | v) - 8388608.f; }

__device__ __forceinline__ float warp_u8(const uint8_t* __restrict__ fr, int pitch, int H, int W, const WorkItem& it,
                                         float cx, float cy, int x, int y) {
  const float dx = (float)x - cx, dy = (float)y - cy;
  const float qx = fmaf(it.a11, dx, fmaf(it.a12, dy, cx));
  const float qy = fmaf(it.a21, dx, fmaf(it.a22, dy, cy));
  const float fx0 = floorf(qx), fy0 = floorf(qy);
  // every tap outside (also keeps the int conversion in range)
  if (!(fx0 >= -1.f && fx0 <= (float)(W - 1) && fy0 >= -1.f && fy0 <= (float)(H - 1))) return 0.f;
  const float fx = qx - fx0, fy = qy - fy0;
  const int x0 = (int)fx0, y0 = (int)fy0;
  const bool xa = x0 >= 0, xb = x0 + 1 < W, ya = y0 >= 0, yb = y0 + 1 < H;
  const uint8_t* r0 = fr + (ya ? y0 : 0) * pitch;
  const uint8_t* r1 = fr + (yb ? y0 + 1 : 0) * pitch;
  const float v00 = (ya && xa) ? u8f(__ldg(r0 + x0)) : 0.f;
  const float v01 = (ya && xb) ? u8f(__ldg(r0 + x0 + 1)) : 0.f;
  const float v10 = (yb && xa) ? u8f(__ldg(r1 + x0)) : 0.f;
  const float v11 = (yb && xb) ? u8f(__ldg(r1 + x0 + 1)) : 0.f;
  const float top = fmaf(fx, v01, (1.f - fx) * v00), bot = fmaf(fx, v11, (1.f - fx) * v10);
  return fmaf(fy, bot, (1.f - fy) * top);
}

// the warped tile with its halo, tile[(ty + 1) * kLTX + tx + 1] = X(x, y)
__device__ __forceinline__ void warp_tile(const uint8_t* __restrict__ frames, size_t pitch, int H, int W,
                                          const WorkItem& it, float* tile) {
  const uint8_t* fr = frames + (size_t)it.frame * H * pitch;
  const float cx = 0.5f * (float)(W - 1), cy = 0.5f * (float)(H - 1);
  const int tid = threadIdx.y * kLX + threadIdx.x;
  const int x0 = blockIdx.x * kLX - 1, y0 = blockIdx.y * kLY - 1;
#pragma unroll
  for (int k0 = 0; k0 < kLTX * kLTY; k0 += kLX * 8) {
    const int k = k0 + tid;
    if (k < kLTX * kLTY) {
      const int sy = k / kLTX, sx = k - sy * kLTX;
      const int y = min(max(y0 + sy, 0), H - 1), x = min(max(x0 + sx, 0), W - 1);
      tile[k] = warp_u8(fr, (int)pitch, H, W, it, cx, cy, x, y);
    }
  }
  __syncthreads();
}

// centre value, window mean offset m1 and population variance of tile pixel (tx, ty)
__device__ __forceinline__ void tile_moments(const float* tile, int tx, int ty, float* xc, float* m1, float* var) {
  const float c = tile[(ty + 1) * kLTX + tx + 1];
  float s1 = 0.f, s2 = 0.f;
#pragma unroll
  for (int dy = 0; dy < 3; ++dy)
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) {
      const float d = tile[(ty + dy) * kLTX + tx + dx] - c;
      s1 += d;
      s2 = fmaf(d, d, s2);
    }
  const float m = s1 * (1.f / 9.f);
  *xc = c;
  *m1 = m;
  *var = fmaf(-m, m, s2 * (1.f / 9.f));
}

// per block: sum of the local variances of its pixels (double), one slot per
// block; the warped frame itself to X[r][H][W] for the second pass
__global__ void __launch_bounds__(kLX * 8) k_lit_moments(const uint8_t* __restrict__ frames, size_t pitch, int H,
                                                         int W, const WorkItem* __restrict__ renders,
                                                         double* __restrict__ partials, float* __restrict__ X) {
  __shared__ float tile[kLTX * kLTY];
  __shared__ double part[8];
  const WorkItem it = renders[blockIdx.z];
  warp_tile(frames, pitch, H, W, it, tile);
  const int tx = threadIdx.x, x = blockIdx.x * kLX + tx;
  if (x < W) {
    float* xo = X + (size_t)blockIdx.z * H * W + x;
#pragma unroll
    for (int k = 0; k < kLR; ++k) {
      const int ty = threadIdx.y + 8 * k, y = blockIdx.y * kLY + ty;
      if (y < H) xo[(size_t)y * W] = tile[(ty + 1) * kLTX + tx + 1];
    }
  }
  // float within a warp (128 terms), double across warps and blocks: the FP64
  // pipe is a small fraction of the FP32 one, so it takes one add per warp
  float v = 0.f;
#pragma unroll
  for (int k = 0; k < kLR; ++k) {
    const int ty = threadIdx.y + 8 * k, y = blockIdx.y * kLY + ty;
    if (x < W && y < H) {
      float c, m, var;
      tile_moments(tile, tx, ty, &c, &m, &var);
      v += var;
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (tx == 0) part[threadIdx.y] = (double)v;
  __syncthreads();
  if (threadIdx.y == 0 && tx == 0) {
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += part[k];
    partials[(size_t)blockIdx.z * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// one block per render: nu2 = (fixed-order sum of the block partials) / (H W)
__global__ void k_lit_noise(const double* __restrict__ partials, int nblk, int H, int W, float* __restrict__ nu2) {
  __shared__ double part[32];
  const int r = blockIdx.x;
  double s = 0.0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) s += partials[(size_t)r * nblk + k];
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += part[k];
    nu2[r] = (float)(t / ((double)H * (double)W));
  }
}

// R of every pixel into out[r * lay.fpitch + lay.roff + y * lay.rpitch + x] (float)
// (the tile and its replicated halo read back from X, the first pass's warped frame)
__global__ void __launch_bounds__(kLX * 8) k_lit_apply(const float* __restrict__ X, int H, int W,
                                                       const float* __restrict__ nu2, int weight,
                                                       float* __restrict__ out, ResidLayout lay) {
  __shared__ float tile[kLTX * kLTY];
  {
    const float* xr = X + (size_t)blockIdx.z * H * W;
    const int tid = threadIdx.y * kLX + threadIdx.x;
    const int x0 = blockIdx.x * kLX - 1, y0 = blockIdx.y * kLY - 1;
#pragma unroll
    for (int k0 = 0; k0 < kLTX * kLTY; k0 += kLX * 8) {
      const int k = k0 + tid;
      if (k < kLTX * kLTY) {
        const int sy = k / kLTX, sx = k - sy * kLTX;
        const int y = min(max(y0 + sy, 0), H - 1), x = min(max(x0 + sx, 0), W - 1);
        tile[k] = __ldg(xr + (size_t)y * W + x);
      }
    }
    __syncthreads();
  }
  const int tx = threadIdx.x, x = blockIdx.x * kLX + tx;
  if (x >= W) return;
  const float n2 = nu2[blockIdx.z];
  float* o = out + (size_t)blockIdx.z * lay.fpitch + lay.roff + x;
#pragma unroll
  for (int k = 0; k < kLR; ++k) {
    const int ty = threadIdx.y + 8 * k, y = blockIdx.y * kLY + ty;
    if (y >= H) break;
    float c, m, var;
    tile_moments(tile, tx, ty, &c, &m, &var);
    const float den = fmaxf(var, n2);
    const float gain = den > 0.f ? __fdividef(fmaxf(var - n2, 0.f), den) : 1.f;
    const float w = -m * (1.f - gain);   // x - (mu + (x - mu) gain), x - mu = -m1
    o[(size_t)y * lay.rpitch] = weight ? c * w : w;
  }
}

// Fingerprint resampling: out(y, x) = sum_a sum_b wy[y][a] wx[x][b] K(iy[y][a], ix[x][b]),
// T taps per axis (unused taps have weight 0 and index 0).
__global__ void k_fp_resize(const float* __restrict__ K, size_t pitch, const float* __restrict__ wy,
                            const int* __restrict__ iy, const float* __restrict__ wx, const int* __restrict__ ix,
                            int T, int H, int W, float* __restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W) return;
  float acc = 0.f;
  for (int a = 0; a < T; ++a) {
    const float w = wy[(size_t)y * T + a];
    if (w == 0.f) continue;
    const float* row = K + (size_t)iy[(size_t)y * T + a] * pitch;
    float r = 0.f;
    for (int b = 0; b < T; ++b) r = fmaf(wx[(size_t)x * T + b], __ldg(row + ix[(size_t)x * T + b]), r);
    acc = fmaf(w, r, acc);
  }
  out[(size_t)y * W + x] = acc;
}

}  // namespace

void launch_fp_estimate_accumulate(const float* R, const uint8_t* frames, size_t pitch, int Lc, int H, int W,
                                   double* num, double* den, bool first, cudaStream_t s, LaunchCounter& lc) {
  ProfScope ps(lc, kKindResidual, s);
  k_fp_accumulate<<<dim3((W + 255) / 256, H), 256, 0, s>>>(R, frames, pitch, Lc, H, W, num, den, first ? 1 : 0);
  PRNU_CUDA_TRY(cudaGetLastError());
  lc.n++;
}

void launch_fp_estimate_divide(const double* num, const double* den, float* K, size_t n, cudaStream_t s,
                               LaunchCounter& lc) {
  ProfScope ps(lc, kKindResidual, s);
  k_fp_divide<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(num, den, K, n);
  PRNU_CUDA_TRY(cudaGetLastError());
  lc.n++;
}

void launch_pad_frames(const void* in, int dtype, int F, int H, int W, void* out, cudaStream_t s, LaunchCounter& lc,
                       int layout) {
  if (F == 0) return;
  ProfScope ps(lc, kKindResidual, s);
  const dim3 b(256), g((W + 3 + 255) / 256, H + 3, F);
  if (layout == 1 && dtype != kF32)
    k_pad_pairs<<<g, b, 0, s>>>(reinterpret_cast<const uint16_t*>(in), H, W, reinterpret_cast<uint32_t*>(out));
  else if (dtype == kF32)
    k_pad_frames<float><<<g, b, 0, s>>>(reinterpret_cast<const float*>(in), H, W, reinterpret_cast<float*>(out));
  else
    k_pad_frames<uint16_t><<<g, b, 0, s>>>(reinterpret_cast<const uint16_t*>(in), H, W,
                                           reinterpret_cast<uint16_t*>(out));
  PRNU_CUDA_TRY(cudaGetLastError());
  lc.n++;
}


void launch_literal_residuals(const uint8_t* frames, size_t pitch, int H, int W, const WorkItem* renders, int nr,
                              int weight, float* out, const ResidLayout& lay, float* X, double* partials,
                              float* nu2, cudaStream_t s, LaunchCounter& lc) {
  if (nr == 0) return;
  ProfScope ps(lc, kKindResidual, s);
  const dim3 b(kLX, 8), g((W + kLX - 1) / kLX, (H + kLY - 1) / kLY, nr);
  k_lit_moments<<<g, b, 0, s>>>(frames, pitch, H, W, renders, partials, X);
  PRNU_CUDA_TRY(cudaGetLastError());
  k_lit_noise<<<nr, 256, 0, s>>>(partials, (int)(g.x * g.y), H, W, nu2);
  PRNU_CUDA_TRY(cudaGetLastError());
  k_lit_apply<<<g, b, 0, s>>>(X, H, W, nu2, weight, out, lay);
  PRNU_CUDA_TRY(cudaGetLastError());
  lc.n += 3;
}

size_t literal_partials_needed(int nr, int H, int W) {
  return (size_t)nr * ((W + kLX - 1) / kLX) * ((H + kLY - 1) / kLY);
}

size_t residual_partials_needed(int F, int H, int W) {
  const size_t gx = (W + kBX - 1) / kBX, gy = (H + kBY - 1) / kBY;
  return (size_t)F * gx * gy;
}

void launch_residual(const uint8_t* frames, int F, int H, int W, size_t pitch, int flags, int dtype, void* out,
                     float* scale, unsigned long long* acc, double* partials, int /*max_partials*/, cudaStream_t s,
                     LaunchCounter& lc, const ResidLayout* lay) {
  const ResidLayout l = lay ? *lay : ResidLayout{W, (size_t)H * W, 0};
  const dim3 b(kBX, 8);
  const dim3 g((W + kBX - 1) / kBX, (H + kBY - 1) / kBY, F);
  const int weight = (flags & PRNU_WEIGHT_BY_INTENSITY) ? 1 : 0;
  ProfScope ps(lc, kKindResidual, s);
  // the block slots go to `partials` (8-byte slots, reused below by PRNU_NORMALISE)
  auto* slots = reinterpret_cast<unsigned long long*>(partials);
  k_resid_moments<<<g, b, 0, s>>>(frames, pitch, H, W, slots);
  PRNU_CUDA_TRY(cudaGetLastError());
  k_resid_noise<<<F, 256, 0, s>>>(slots, (int)(g.x * g.y), acc);
  PRNU_CUDA_TRY(cudaGetLastError());
  lc.n += 2;
  if (flags & PRNU_NORMALISE) {
    apply_dispatch<1>(dtype, g, b, s, frames, pitch, H, W, acc, weight, out, partials, scale, l);
    PRNU_CUDA_TRY(cudaGetLastError());
    k_resid_scale<<<F, 256, 0, s>>>(partials, (int)(g.x * g.y), H, W, scale);
    PRNU_CUDA_TRY(cudaGetLastError());
    apply_dispatch<2>(dtype, g, b, s, frames, pitch, H, W, acc, weight, out, partials, scale, l);
    PRNU_CUDA_TRY(cudaGetLastError());
    lc.n += 3;
  } else {
    apply_dispatch<0>(dtype, g, b, s, frames, pitch, H, W, acc, weight, out, partials, scale, l);
    PRNU_CUDA_TRY(cudaGetLastError());
    lc.n++;
    if (scale) {
      k_fill<<<(F + 255) / 256, 256, 0, s>>>(scale, F, 1.f);
      PRNU_CUDA_TRY(cudaGetLastError());
      lc.n++;
    }
  }
}

}  // namespace prnu

namespace prnu {
void launch_fp_resize(const float* K, size_t pitch, const float* wy, const int* iy, const float* wx, const int* ix,
                      int T, int H, int W, float* out, cudaStream_t s, LaunchCounter& lc) {
  ProfScope ps(lc, kKindResidual, s);
  k_fp_resize<<<dim3((W + 127) / 128, H), 128, 0, s>>>(K, pitch, wy, iy, wx, ix, T, H, W, out);
  PRNU_CUDA_TRY(cudaGetLastError());
  lc.n++;
}
}  // namespace prnu

namespace prnu {
void launch_resid_scale(const double* partials, int nblk, int F, int H, int W, float* scale, cudaStream_t s,
                        LaunchCounter& lc) {
  k_resid_scale<<<F, 256, 0, s>>>(partials, nblk, H, W, scale);
  PRNU_CUDA_TRY(cudaGetLastError());
  lc.n++;
}
void launch_fill(float* p, int n, float v, cudaStream_t s, LaunchCounter& lc) {
  k_fill<<<(n + 255) / 256, 256, 0, s>>>(p, n, v);
  PRNU_CUDA_TRY(cudaGetLastError());
  lc.n++;
}
}  // namespace prnu
