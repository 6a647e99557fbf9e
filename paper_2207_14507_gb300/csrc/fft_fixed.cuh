// fft_fixed.cuh -- Stockham FFT stages with a compile-time plan.
//
// The autosort stage of fft.cuh (stage with radix R, Ns = product of the
// earlier radices: butterfly j reads x[j + r*n/R], twiddles input r by
// w_{Ns*R}^{r*(j mod Ns)}, writes output r to y[(j/Ns)*Ns*R + (j mod Ns) + r*Ns]),
// with n, R, Ns and the thread count known at compile time and the shared
// memory layouts chosen so that every element a thread touches lies at a
// compile-time offset from one per-thread base address:
//
//  * row layout (one transform per thread group): element i at
//    i + 2*floor(i/16).  With a first radix of 16 and n/R and Ns multiples of
//    16 in the later stages, the loads j + r*n/R and stores base + r*Ns move
//    by whole 16-element blocks, so each is base + constant.  The two float2
//    of padding per 16 keep the stride-18 stores of the first stage and the
//    unit-stride loads of the next one free of bank conflicts, and keep every
//    even element 16-byte aligned, so the first stage stores pairs of outputs
//    with one 16-byte store.
//  * column layout (NC interleaved transforms): element i of column c at
//    i*NC + c, unpadded; a thread owns a pair of adjacent columns, so every
//    shared and global access is a 16-byte vector and the two columns share
//    one set of twiddles.
//
// Stage twiddles come from per-stage tables evaluated at compile time in
// double precision with an exact argument reduction and rounded to float; a
// butterfly reads its R-1 twiddles as 16-byte pairs at constant offsets from
// one base address, the pairs of neighbouring butterflies adjacent.
#pragma once
#include <type_traits>

#include "fft.cuh"

namespace prnu {

template <int N_, int R0, int R1 = 1, int R2 = 1, int R3 = 1>
struct Spec {
  static constexpr int N = N_;
  static constexpr int S = (R1 == 1) ? 1 : (R2 == 1) ? 2 : (R3 == 1) ? 3 : 4;
  __host__ __device__ static constexpr int r(int i) { return i == 0 ? R0 : i == 1 ? R1 : i == 2 ? R2 : R3; }
  __host__ __device__ static constexpr int ns(int i) { return i == 0 ? 1 : ns(i - 1) * r(i - 1); }
  static_assert(R0 * R1 * R2 * R3 == N_, "radices must multiply to N");
  // the reversed plan: the inverse transform that follows a forward one
  using Rev = typename std::conditional<
      S == 1, Spec<N_, R0>,
      typename std::conditional<
          S == 2, Spec<N_, R1, R0>,
          typename std::conditional<S == 3, Spec<N_, R2, R1, R0>, Spec<N_, R3, R2, R1, R0>>::type>::type>::type;
};

// stage I of plan SP
template <class SP, int I>
struct Stg {
  static constexpr int N = SP::N;
  static constexpr int R = SP::r(I);
  static constexpr int NS = SP::ns(I);
  static constexpr int NB = N / R;   // butterflies
};

// ---------------------------------------------------------------- compile-time twiddles

// Series for |x| <= pi/4; a term is dropped once it is below 1e-100, so no
// step underflows (constant evaluation rejects subnormal results).
__host__ __device__ constexpr double ce_sin_small(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 16; ++k) {
    term *= -x * x / double((2 * k) * (2 * k + 1));
    if (term < 1e-100 && term > -1e-100) break;
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double ce_cos_small(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 16; ++k) {
    term *= -x * x / double((2 * k - 1) * (2 * k));
    if (term < 1e-100 && term > -1e-100) break;
    sum += term;
  }
  return sum;
}

struct CeCosSin {
  double c, s;
};
// cos and sin of 2*pi*m/n, reduced exactly in integers to an angle pi*p/q in
// [0, pi/4] (quadrant and octant symmetries), so multiples of pi/4 are exact.
__host__ __device__ constexpr CeCosSin ce_cossin2pi(long m, long n) {
  long p = ((m % n) + n) % n * 2, q = n;        // angle pi*p/q, p in [0, 2q)
  double sgs = 1.0, sgc = 1.0;
  if (p > q) {                                  // (pi, 2pi): sin(2pi - a) = -sin a
    p = 2 * q - p;
    sgs = -1.0;
  }
  if (2 * p > q) {                              // (pi/2, pi]: cos(pi - a) = -cos a
    p = q - p;
    sgc = -1.0;
  }
  bool swap = false;
  if (4 * p > q) {                              // (pi/4, pi/2]: cos a = sin(pi/2 - a)
    p = q - 2 * p;
    q = 2 * q;
    swap = true;
  }
  const double x = 3.14159265358979323846264338327950288 * double(p) / double(q);
  const double c = ce_cos_small(x), s = ce_sin_small(x);
  return CeCosSin{sgc * (swap ? s : c), sgs * (swap ? c : s)};
}

// Twiddles of one stage, w_{Ns*R}^{r*k} (forward, w = exp(-2 pi i / n)) for
// k < Ns, 1 <= r < R, in pairs: entry (m, k) = (w^{(2m+1)k}, w^{(2m+2)k}) as
// one float4 at v[4*(m*Ns + k)], m < RP/2 (RP = R - 1 rounded up to even;
// a pair past r = R - 1 is zero).  Consecutive k are adjacent, so the
// threads of a warp, which hold consecutive k, read whole cache lines.
template <int R, int NS>
struct TwTab {
  static constexpr int RP = (R & 1) ? R - 1 : R;
  alignas(16) float v[2 * NS * RP];
};
template <int R, int NS>
constexpr TwTab<R, NS> make_twtab() {
  TwTab<R, NS> t{};
  for (int m = 0; m < TwTab<R, NS>::RP / 2; ++m)
    for (int k = 0; k < NS; ++k)
      for (int h = 0; h < 2; ++h) {
        const int r = 2 * m + 1 + h;
        if (r >= R) continue;
        const CeCosSin w = ce_cossin2pi((long)r * k, (long)NS * R);
        t.v[4 * (m * NS + k) + 2 * h] = float(w.c);
        t.v[4 * (m * NS + k) + 2 * h + 1] = float(-w.s);
      }
  return t;
}
template <int R, int NS>
__device__ constexpr TwTab<R, NS> kStageTw = make_twtab<R, NS>();

// v * w (forward) or v * conj(w) (INV), w = (wx, wy), with the rounding fixed
// (one product rounded on its own plus one fused multiply-add per component)
// so that every kernel running a stage gets the same bits.
template <bool INV>
__device__ __forceinline__ float2 tw_mul(float2 v, float wx, float wy) {
  return INV ? make_float2(__fmaf_rn(v.x, wx, __fmul_rn(v.y, wy)), __fmaf_rn(v.y, wx, -__fmul_rn(v.x, wy)))
             : make_float2(__fmaf_rn(v.x, wx, -__fmul_rn(v.y, wy)), __fmaf_rn(v.x, wy, __fmul_rn(v.y, wx)));
}

// v[n][r] *= w_{Ns*R}^{r*k} (conjugate for INV) for the NV transforms of one
// butterfly position (they share k); nothing for Ns = 1.
template <int R, int NS, bool INV, int NV>
__device__ __forceinline__ void twiddle_tab(float2 (&v)[NV][R], int k) {
  if constexpr (NS > 1) {
    constexpr int RP = TwTab<R, NS>::RP;
    const float4* p = reinterpret_cast<const float4*>(kStageTw<R, NS>.v) + k;
#pragma unroll
    for (int m = 0; m < RP / 2; ++m) {
      const float4 w = __ldg(p + m * NS);
      const int r = 2 * m + 1;
#pragma unroll
      for (int n = 0; n < NV; ++n) v[n][r] = tw_mul<INV>(v[n][r], w.x, w.y);
      if (r + 1 < R) {
#pragma unroll
        for (int n = 0; n < NV; ++n) v[n][r + 1] = tw_mul<INV>(v[n][r + 1], w.z, w.w);
      }
    }
  }
}

// ---------------------------------------------------------------- row layout

__host__ __device__ constexpr int rp2(int i) { return i + 2 * (i >> 4); }
__host__ __device__ constexpr int row_len2(int n) { return n + n / 8; }

// Stage 0 output store of a radix-16 first stage (Ns = 1): outputs j*16 + r at
// 18*j + r, as eight 16-byte pairs.
__device__ __forceinline__ void row_store16(float2* out, int j, const float2 (&v)[16]) {
  float4* d = reinterpret_cast<float4*>(out + 18 * j);
#pragma unroll
  for (int m = 0; m < 8; ++m) d[m] = make_float4(v[2 * m].x, v[2 * m].y, v[2 * m + 1].x, v[2 * m + 1].y);
}

// Stage I (>= 1) of row plan SP on one transform, T threads (thread t),
// in -> out, both in the row layout.
template <class SP, int I, int T, bool INV>
__device__ __forceinline__ void row_stage(const float2* __restrict__ in, float2* __restrict__ out, int t) {
  using G = Stg<SP, I>;
  static_assert(G::NB % 16 == 0 && G::NS % 16 == 0 && T % 16 == 0, "row stages need 16-element blocks");
  constexpr int IT = (G::NB + T - 1) / T;
  constexpr int LB = G::NB / 16 * 18, LS = G::NS / 16 * 18;
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int j = t + it * T;
    if (G::NB % T != 0 && j >= G::NB) break;
    float2 v[1][G::R];
    const float2* src = in + rp2(j);
#pragma unroll
    for (int r = 0; r < G::R; ++r) v[0][r] = src[r * LB];
    const int k = (G::NB == G::NS) ? j : j % G::NS;
    twiddle_tab<G::R, G::NS, INV, 1>(v, k);
    Dft<G::R, INV>::run(v[0]);
    float2* dst = out + rp2((j - k) * G::R + k);
#pragma unroll
    for (int r = 0; r < G::R; ++r) dst[r * LS] = v[0][r];
  }
}

// Stage I (>= 1) of row plan SP in place on `buf`, one butterfly per thread
// (NB <= T): every thread loads its inputs, the block synchronises, then every
// thread stores its outputs.  One row buffer instead of two, for one more
// barrier.  Called by every thread of the block.
template <class SP, int I, int T, bool INV>
__device__ __forceinline__ void row_stage_ip(float2* buf, int t) {
  using G = Stg<SP, I>;
  static_assert(G::NB % 16 == 0 && G::NS % 16 == 0 && T % 16 == 0, "row stages need 16-element blocks");
  static_assert(G::NB <= T, "in-place row stages hold one butterfly per thread");
  constexpr int LB = G::NB / 16 * 18, LS = G::NS / 16 * 18;
  const bool act = G::NB == T || t < G::NB;
  const int j = t;
  const int k = (G::NB == G::NS) ? j : j % G::NS;
  float2 v[1][G::R];
  if (act) {
    const float2* src = buf + rp2(j);
#pragma unroll
    for (int r = 0; r < G::R; ++r) v[0][r] = src[r * LB];
  }
  __syncthreads();
  if (act) {
    twiddle_tab<G::R, G::NS, INV, 1>(v, k);
    Dft<G::R, INV>::run(v[0]);
    float2* dst = buf + rp2((j - k) * G::R + k);
#pragma unroll
    for (int r = 0; r < G::R; ++r) dst[r * LS] = v[0][r];
  }
}

// Last stage of row plan SP (Ns = n/R): butterflies j = t + it*T, outputs
// x = j + r*Ns stay in registers, v[it]; `last_valid` tells which are real.
template <class SP, int T>
struct RowLast {
  using G = Stg<SP, SP::S - 1>;
  static constexpr int R = G::R;
  static constexpr int NS = G::NS;
  static constexpr int IT = (G::NB + T - 1) / T;
  static_assert(G::NB == G::NS && G::NB % 16 == 0, "last stage: k = j");
  __device__ __forceinline__ static bool valid(int t, int it) { return G::NB % T == 0 || t + it * T < G::NB; }
};

template <class SP, int T, bool INV>
__device__ __forceinline__ void row_stage_last(const float2* __restrict__ in, int t,
                                               float2 (&v)[RowLast<SP, T>::IT][RowLast<SP, T>::R]) {
  using L = RowLast<SP, T>;
  constexpr int LB = L::NS / 16 * 18;
#pragma unroll
  for (int it = 0; it < L::IT; ++it) {
    if (!L::valid(t, it)) break;
    const int j = t + it * T;
    const float2* src = in + rp2(j);
    float2 u[1][L::R];
#pragma unroll
    for (int r = 0; r < L::R; ++r) u[0][r] = src[r * LB];
    twiddle_tab<L::R, L::NS, INV, 1>(u, j);
    Dft<L::R, INV>::run(u[0]);
#pragma unroll
    for (int r = 0; r < L::R; ++r) v[it][r] = u[0][r];
  }
}

// ---------------------------------------------------------------- column layout

// Threads -> (butterfly row j, column pair cp): cp = t % NP, j = t / NP + it * (T / NP).
template <int NC, int T>
struct ColMap {
  static constexpr int NP = NC / 2;
  static constexpr int TJ = T / NP;
  static_assert(NC % 2 == 0 && T % NP == 0, "a thread owns a pair of columns");
};

__device__ __forceinline__ void split2(float4 q, float2& a, float2& b) {
  a = make_float2(q.x, q.y);
  b = make_float2(q.z, q.w);
}
__device__ __forceinline__ float4 join2(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

// In-place middle stage I of column plan SP (NC columns, T threads): load
// everything, barrier, transform, store, barrier.
template <class SP, int I, int T, int NC, bool INV>
__device__ __forceinline__ void col_stage_ip(float4* sm4, int t) {
  using G = Stg<SP, I>;
  using M = ColMap<NC, T>;
  constexpr int IT = (G::NB + M::TJ - 1) / M::TJ;
  const int cp = t % M::NP, j0 = t / M::NP;
  float2 v[IT][2][G::R];
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int j = j0 + it * M::TJ;
    if (G::NB % M::TJ != 0 && j >= G::NB) continue;
    const float4* src = sm4 + j * M::NP + cp;
#pragma unroll
    for (int r = 0; r < G::R; ++r) split2(src[r * G::NB * M::NP], v[it][0][r], v[it][1][r]);
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int j = j0 + it * M::TJ;
    if (G::NB % M::TJ != 0 && j >= G::NB) continue;
    const int k = j % G::NS;
    twiddle_tab<G::R, G::NS, INV, 2>(v[it], k);
    Dft<G::R, INV>::run(v[it][0]);
    Dft<G::R, INV>::run(v[it][1]);
    float4* dst = sm4 + ((j - k) * G::R + k) * M::NP + cp;
#pragma unroll
    for (int r = 0; r < G::R; ++r) dst[r * G::NS * M::NP] = join2(v[it][0][r], v[it][1][r]);
  }
  __syncthreads();
}

template <class SP, int I, int I1, int T, int NC, bool INV>
struct ColStages {
  __device__ __forceinline__ static void run(float4* sm4, int t) {
    if constexpr (I < I1) {
      col_stage_ip<SP, I, T, NC, INV>(sm4, t);
      ColStages<SP, I + 1, I1, T, NC, INV>::run(sm4, t);
    }
  }
};

}  // namespace prnu
