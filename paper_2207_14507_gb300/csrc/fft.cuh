// fft.cuh -- block-level mixed-radix FFT engine (device code).
//
// A length-n complex FFT (n = 2^a 3^b 5^c) runs in shared memory as a
// sequence of Stockham autosort stages (Govindaraju et al., SC'08 formulation):
// stage s with radix R and Ns = product of the previous radices reads, for
// butterfly j < n/R, the R inputs x[j + r*n/R], multiplies input r by
// w_{Ns*R}^{r*(j mod Ns)}, takes a length-R DFT in registers and writes output r
// to y[(j/Ns)*Ns*R + (j mod Ns) + r*Ns].
//
// The in-register DFTs of size R in {2,3,4,5,6,8,9,10,12,15,16} are built at
// compile time: sizes 2..5 from their closed forms, the others by a two-factor
// Cooley-Tukey split R = P*Q whose inner twiddles are compile-time constants.
// Those constants come from a constexpr Taylor series (they are only ever
// w_R^k for R <= 16); the stage twiddles w_n^k come from a table the host
// builds in double precision and rounds to float.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <type_traits>

namespace prnu {

// ---------------------------------------------------------------- compile-time roots of unity

__host__ __device__ constexpr double ce_pi() { return 3.14159265358979323846264338327950288; }

// Taylor series, |x| <= pi/2 after reduction: 14 terms reach double rounding.
__host__ __device__ constexpr double ce_sin_poly(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 14; ++k) {
    term *= -x * x / double((2 * k) * (2 * k + 1));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double ce_cos_poly(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 14; ++k) {
    term *= -x * x / double((2 * k - 1) * (2 * k));
    sum += term;
  }
  return sum;
}
// cos and sin of 2*pi*m/n for integers m, n > 0.
__host__ __device__ constexpr double ce_cos2pi(long m, long n) {
  long r = ((m % n) + n) % n;
  if (2 * r > n) r -= n;                       // angle in (-pi, pi]
  double a = 2.0 * ce_pi() * double(r) / double(n);
  double aa = a < 0 ? -a : a;
  if (aa > ce_pi() / 2) return -ce_cos_poly(ce_pi() - aa);
  return ce_cos_poly(aa);
}
__host__ __device__ constexpr double ce_sin2pi(long m, long n) {
  long r = ((m % n) + n) % n;
  if (2 * r > n) r -= n;
  double a = 2.0 * ce_pi() * double(r) / double(n);
  double sg = a < 0 ? -1.0 : 1.0;
  double aa = a < 0 ? -a : a;
  if (aa > ce_pi() / 2) return sg * ce_sin_poly(ce_pi() - aa);
  return sg * ce_sin_poly(aa);
}

// ---------------------------------------------------------------- complex helpers

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ float2 c_mulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }
// conj(a) * b with its rounding fixed: each component is one product rounded
// on its own plus one fused multiply-add, so every kernel that forms this
// product gets the same bits (no contraction left to the compiler's choice).
__device__ __forceinline__ float2 c_conj_mul(float2 a, float2 b) {
  return make_float2(__fmaf_rn(a.x, b.x, __fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, -__fmul_rn(a.y, b.x)));
}
// multiply by -i (forward quarter turn) / +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 c_quarter(float2 v) {
  return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
}

// v * w_N^M with w_N = exp(-2 pi i / N) (forward) or exp(+2 pi i / N) (inverse),
// M and N compile-time; exact quarter turns are done by swaps.
template <int M, int N, bool INV>
__device__ __forceinline__ float2 c_twiddle(float2 v) {
  constexpr int m = ((M % N) + N) % N;
  if constexpr (m == 0) {
    return v;
  } else if constexpr (2 * m == N) {
    return make_float2(-v.x, -v.y);
  } else if constexpr (4 * m == N) {
    return c_quarter<INV>(v);
  } else if constexpr (4 * m == 3 * N) {
    return c_quarter<!INV>(v);
  } else {
    constexpr float c = float(ce_cos2pi(m, N));
    constexpr float s = float(INV ? ce_sin2pi(m, N) : -ce_sin2pi(m, N));
    return make_float2(v.x * c - v.y * s, v.x * s + v.y * c);
  }
}

// ---------------------------------------------------------------- in-register DFTs

template <int R>
struct FirstFactor {
  static constexpr int value = (R % 4 == 0 && R != 4 && R != 8) ? 4 : (R % 2 == 0 ? 2 : (R % 3 == 0 ? 3 : 5));
};

template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
  __device__ __forceinline__ static void run(float2 (&x)[2]) {
    float2 a = x[0], b = x[1];
    x[0] = c_add(a, b);
    x[1] = c_sub(a, b);
  }
};

template <bool INV>
struct Dft<3, INV> {
  __device__ __forceinline__ static void run(float2 (&x)[3]) {
    constexpr float h = 0.8660254037844386f;  // sin(2 pi / 3)
    float2 a = x[0];
    float2 t = c_add(x[1], x[2]);
    float2 u = c_sub(x[1], x[2]);
    float2 m = make_float2(a.x - 0.5f * t.x, a.y - 0.5f * t.y);
    // forward: X1 = m - i h u, X2 = m + i h u
    float2 ihu = INV ? make_float2(-h * u.y, h * u.x) : make_float2(h * u.y, -h * u.x);
    x[0] = c_add(a, t);
    x[1] = c_add(m, ihu);
    x[2] = c_sub(m, ihu);
  }
};

template <bool INV>
struct Dft<4, INV> {
  __device__ __forceinline__ static void run(float2 (&x)[4]) {
    float2 s02 = c_add(x[0], x[2]), d02 = c_sub(x[0], x[2]);
    float2 s13 = c_add(x[1], x[3]), d13 = c_quarter<INV>(c_sub(x[1], x[3]));
    x[0] = c_add(s02, s13);
    x[2] = c_sub(s02, s13);
    x[1] = c_add(d02, d13);
    x[3] = c_sub(d02, d13);
  }
};

template <bool INV>
struct Dft<5, INV> {
  __device__ __forceinline__ static void run(float2 (&x)[5]) {
    constexpr float c1 = float(ce_cos2pi(1, 5)), c2 = float(ce_cos2pi(2, 5));
    constexpr float s1 = float(ce_sin2pi(1, 5)), s2 = float(ce_sin2pi(2, 5));
    float2 a = x[0];
    float2 t1 = c_add(x[1], x[4]), t2 = c_add(x[2], x[3]);
    float2 t3 = c_sub(x[1], x[4]), t4 = c_sub(x[2], x[3]);
    float2 m1 = make_float2(a.x + c1 * t1.x + c2 * t2.x, a.y + c1 * t1.y + c2 * t2.y);
    float2 m2 = make_float2(a.x + c2 * t1.x + c1 * t2.x, a.y + c2 * t1.y + c1 * t2.y);
    float2 n1 = make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y);
    float2 n2 = make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y);
    // forward: X1 = m1 - i n1, X4 = m1 + i n1, X2 = m2 - i n2, X3 = m2 + i n2
    float2 q1 = c_quarter<INV>(n1), q2 = c_quarter<INV>(n2);
    x[0] = make_float2(a.x + t1.x + t2.x, a.y + t1.y + t2.y);
    x[1] = c_add(m1, q1);
    x[4] = c_sub(m1, q1);
    x[2] = c_add(m2, q2);
    x[3] = c_sub(m2, q2);
  }
};

// Composite R = P*Q: n = Q*n1 + n2, k = k1 + P*k2;
// X[k1 + P k2] = sum_n2 w_Q^{n2 k2} w_R^{n2 k1} sum_n1 x[Q n1 + n2] w_P^{n1 k1}.
// The compile-time index loops are forced-inline template recursions so that
// every array stays in registers.
template <int R, bool INV, int P, int N2, int K1>
struct CompTwiddle {
  __device__ __forceinline__ static void run(const float2 (&t)[P], float2 (&y)[R]) {
    if constexpr (K1 < P) {
      y[N2 * P + K1] = c_twiddle<N2 * K1, R, INV>(t[K1]);
      CompTwiddle<R, INV, P, N2, K1 + 1>::run(t, y);
    }
  }
};

template <int R, bool INV, int P, int Q, int N2>
struct CompInner {
  __device__ __forceinline__ static void run(const float2 (&x)[R], float2 (&y)[R]) {
    if constexpr (N2 < Q) {
      float2 t[P];
#pragma unroll
      for (int n1 = 0; n1 < P; ++n1) t[n1] = x[Q * n1 + N2];
      Dft<P, INV>::run(t);
      CompTwiddle<R, INV, P, N2, 0>::run(t, y);
      CompInner<R, INV, P, Q, N2 + 1>::run(x, y);
    }
  }
};

template <int R, bool INV>
struct Dft {
  static constexpr int P = FirstFactor<R>::value;
  static constexpr int Q = R / P;
  __device__ __forceinline__ static void run(float2 (&x)[R]) {
    float2 y[R];
    CompInner<R, INV, P, Q, 0>::run(x, y);
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      float2 t[Q];
#pragma unroll
      for (int n2 = 0; n2 < Q; ++n2) t[n2] = y[n2 * P + k1];
      Dft<Q, INV>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) x[k1 + P * k2] = t[k2];
    }
  }
};

// ---------------------------------------------------------------- plans

constexpr int kMaxStages = 8;
constexpr int kMaxFft = 4096;

// A length-n plan: radices in execution order and the offset of the w_n^k
// table (n entries) inside the context's twiddle buffer.
struct FftPlan {
  int n;
  int nstages;
  int radix[kMaxStages];
  int tw_off;
  int min_radix;
};

// ---------------------------------------------------------------- stages
//
// Stages run out of place between two shared-memory buffers (ping-pong): a
// thread loads one butterfly's R inputs, transforms them in registers and
// stores the R outputs before it takes the next butterfly, so no register
// state crosses a barrier.  Two layouts:
//  * row layout: one FFT per thread group, element i at i + (i >> 4) (one
//    float2 of padding every 16 keeps the strided stores off one bank);
//  * column layout: NC = 1 << lg interleaved FFTs (columns), element i of
//    column c at i*NC + c; butterflies are spread over all threads of the block.

__device__ __forceinline__ int rpad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int row_smem_len(int n) { return n + (n >> 4) + 1; }

template <int R, bool INV>
__device__ __forceinline__ void twiddle_inputs(float2 (&v)[R], int k, int step_unit,
                                               const float2* __restrict__ tw) {
  // v[r] *= w_n^{r * k * step_unit}, step_unit = n / (Ns * R)
  if (k == 0) return;
  const int s = k * step_unit;
#pragma unroll
  for (int r = 1; r < R; ++r) {
    float2 w = __ldg(tw + r * s);
    v[r] = INV ? c_mulc(v[r], w) : c_mul(v[r], w);
  }
}

template <int R, bool INV>
__device__ __forceinline__ void stage_row(const float2* __restrict__ in, float2* __restrict__ out, int n, int ns,
                                          const float2* __restrict__ tw, int t, int T) {
  const int nb = n / R;
  const int unit = n / (ns * R);
  for (int j = t; j < nb; j += T) {
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[rpad(j + r * nb)];
    const int k = j % ns;
    twiddle_inputs<R, INV>(v, k, unit, tw);
    Dft<R, INV>::run(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) out[rpad(base + r * ns)] = v[r];
  }
}

template <int R, bool INV>
__device__ __forceinline__ void stage_col(const float2* __restrict__ in, float2* __restrict__ out, int n, int ns,
                                          const float2* __restrict__ tw, int t, int T, int lg) {
  const int nb = n / R;
  const int unit = n / (ns * R);
  const int total = nb << lg;
  const int cm = (1 << lg) - 1;
  for (int g = t; g < total; g += T) {
    const int j = g >> lg, c = g & cm;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[((j + r * nb) << lg) + c];
    const int k = j % ns;
    twiddle_inputs<R, INV>(v, k, unit, tw);
    Dft<R, INV>::run(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) out[((base + r * ns) << lg) + c] = v[r];
  }
}

// Full FFT of the data in `a` (row layout), using `b` as the second buffer.
// Every thread of the block must call it (it holds barriers); a thread of a
// group without a row passes t >= n so that it owns no butterfly.  The caller
// synchronises before the call; the result is in the returned buffer and is
// visible to the whole block on return.
template <bool INV>
__device__ float2* fft_row(float2* a, float2* b, const FftPlan& p, const float2* __restrict__ twtab, int t, int T) {
  const float2* tw = twtab + p.tw_off;
  int ns = 1;
  for (int s = 0; s < p.nstages; ++s) {
    const int R = p.radix[s];
    switch (R) {
      case 2: stage_row<2, INV>(a, b, p.n, ns, tw, t, T); break;
      case 3: stage_row<3, INV>(a, b, p.n, ns, tw, t, T); break;
      case 4: stage_row<4, INV>(a, b, p.n, ns, tw, t, T); break;
      case 5: stage_row<5, INV>(a, b, p.n, ns, tw, t, T); break;
      case 6: stage_row<6, INV>(a, b, p.n, ns, tw, t, T); break;
      case 8: stage_row<8, INV>(a, b, p.n, ns, tw, t, T); break;
      case 9: stage_row<9, INV>(a, b, p.n, ns, tw, t, T); break;
      case 10: stage_row<10, INV>(a, b, p.n, ns, tw, t, T); break;
      case 12: stage_row<12, INV>(a, b, p.n, ns, tw, t, T); break;
      case 15: stage_row<15, INV>(a, b, p.n, ns, tw, t, T); break;
      default: stage_row<16, INV>(a, b, p.n, ns, tw, t, T); break;
    }
    __syncthreads();
    float2* x = a;
    a = b;
    b = x;
    ns *= R;
  }
  return a;
}

template <bool INV>
__device__ float2* fft_col(float2* a, float2* b, const FftPlan& p, const float2* __restrict__ twtab, int t, int T,
                           int lg) {
  const float2* tw = twtab + p.tw_off;
  int ns = 1;
  for (int s = 0; s < p.nstages; ++s) {
    const int R = p.radix[s];
    switch (R) {
      case 2: stage_col<2, INV>(a, b, p.n, ns, tw, t, T, lg); break;
      case 3: stage_col<3, INV>(a, b, p.n, ns, tw, t, T, lg); break;
      case 4: stage_col<4, INV>(a, b, p.n, ns, tw, t, T, lg); break;
      case 5: stage_col<5, INV>(a, b, p.n, ns, tw, t, T, lg); break;
      case 6: stage_col<6, INV>(a, b, p.n, ns, tw, t, T, lg); break;
      case 8: stage_col<8, INV>(a, b, p.n, ns, tw, t, T, lg); break;
      case 9: stage_col<9, INV>(a, b, p.n, ns, tw, t, T, lg); break;
      case 10: stage_col<10, INV>(a, b, p.n, ns, tw, t, T, lg); break;
      case 12: stage_col<12, INV>(a, b, p.n, ns, tw, t, T, lg); break;
      case 15: stage_col<15, INV>(a, b, p.n, ns, tw, t, T, lg); break;
      default: stage_col<16, INV>(a, b, p.n, ns, tw, t, T, lg); break;
    }
    __syncthreads();
    float2* x = a;
    a = b;
    b = x;
    ns *= R;
  }
  return a;
}

}  // namespace prnu
