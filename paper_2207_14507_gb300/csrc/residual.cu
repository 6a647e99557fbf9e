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

constexpr int kBX = 32, kBY = 8;

__device__ __forceinline__ void moments3x3(const uint8_t* __restrict__ f, size_t pitch, int H, int W, int y, int x,
                                           int* s1, int* s2, int* xc) {
  int a = 0, b = 0;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
    int yy = min(max(y + dy, 0), H - 1);
    const uint8_t* row = f + (size_t)yy * pitch;
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      int xx = min(max(x + dx, 0), W - 1);
      int v = __ldg(row + xx);
      a += v;
      b += v * v;
    }
  }
  *s1 = a;
  *s2 = b;
  *xc = __ldg(f + (size_t)y * pitch + x);
}

__global__ void k_resid_moments(const uint8_t* __restrict__ frames, size_t pitch, int H, int W,
                                unsigned long long* __restrict__ acc) {
  __shared__ unsigned long long part[kBX * kBY / 32];
  const int f = blockIdx.z;
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  const uint8_t* fr = frames + (size_t)f * H * pitch;
  unsigned long long v = 0;
  if (x < W && y < H) {
    int s1, s2, xc;
    moments3x3(fr, pitch, H, W, y, x, &s1, &s2, &xc);
    v = (unsigned long long)(9 * s2 - s1 * s1);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int tid = threadIdx.y * kBX + threadIdx.x;
  if ((tid & 31) == 0) part[tid >> 5] = v;
  __syncthreads();
  if (tid == 0) {
    unsigned long long s = 0;
    for (int k = 0; k < kBX * kBY / 32; ++k) s += part[k];
    if (s) atomicAdd(acc + f, s);
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
__global__ void k_resid_apply(const uint8_t* __restrict__ frames, size_t pitch, int H, int W,
                              const unsigned long long* __restrict__ acc, int weight, void* __restrict__ out,
                              double* __restrict__ partials, const float* __restrict__ scale, ResidLayout lay) {
  __shared__ double part[kBX * kBY / 32];
  const int f = blockIdx.z;
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  const uint8_t* fr = frames + (size_t)f * H * pitch;
  const double nu2d = (double)acc[f] / (81.0 * (double)H * (double)W);
  const float nu2 = (float)nu2d;
  const float nu2x81 = (float)(81.0 * nu2d);
  float r = 0.f;
  if (x < W && y < H) {
    int s1, s2, xc;
    moments3x3(fr, pitch, H, W, y, x, &s1, &s2, &xc);
    r = residual_value(s1, s2, xc, nu2, nu2x81, weight);
    const size_t o = (size_t)f * lay.fpitch + lay.roff + (size_t)y * lay.rpitch + x;
    if (MODE == 0) store_store_type<DT>(out, o, r);
    if (MODE == 2) store_store_type<DT>(out, o, r * scale[f]);
  }
  if (MODE == 1) {
    double v = (double)r * (double)r;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int tid = threadIdx.y * kBX + threadIdx.x;
    if ((tid & 31) == 0) part[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      double s = 0;
      for (int k = 0; k < kBX * kBY / 32; ++k) s += part[k];
      partials[(size_t)f * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = s;
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

void launch_pad_frames(const void* in, int dtype, int F, int H, int W, void* out, cudaStream_t s, LaunchCounter& lc) {
  if (F == 0) return;
  ProfScope ps(lc, kKindResidual, s);
  const dim3 b(256), g((W + 3 + 255) / 256, H + 3, F);
  if (dtype == kF32)
    k_pad_frames<float><<<g, b, 0, s>>>(reinterpret_cast<const float*>(in), H, W, reinterpret_cast<float*>(out));
  else
    k_pad_frames<uint16_t><<<g, b, 0, s>>>(reinterpret_cast<const uint16_t*>(in), H, W,
                                           reinterpret_cast<uint16_t*>(out));
  PRNU_CUDA_TRY(cudaGetLastError());
  lc.n++;
}

size_t residual_partials_needed(int F, int H, int W) {
  const size_t gx = (W + kBX - 1) / kBX, gy = (H + kBY - 1) / kBY;
  return (size_t)F * gx * gy;
}

void launch_residual(const uint8_t* frames, int F, int H, int W, size_t pitch, int flags, int dtype, void* out,
                     float* scale, unsigned long long* acc, double* partials, int /*max_partials*/, cudaStream_t s,
                     LaunchCounter& lc, const ResidLayout* lay) {
  const ResidLayout l = lay ? *lay : ResidLayout{W, (size_t)H * W, 0};
  const dim3 b(kBX, kBY);
  const dim3 g((W + kBX - 1) / kBX, (H + kBY - 1) / kBY, F);
  const int weight = (flags & PRNU_WEIGHT_BY_INTENSITY) ? 1 : 0;
  ProfScope ps(lc, kKindResidual, s);
  PRNU_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * F, s));
  k_resid_moments<<<g, b, 0, s>>>(frames, pitch, H, W, acc);
  PRNU_CUDA_TRY(cudaGetLastError());
  lc.n++;
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
