// fft_fixed.cuh -- Stockham FFT stages with a compile-time plan.
//
// The same autosort stage as fft.cuh (stage with radix R, Ns = product of the
// earlier radices: butterfly j reads x[j + r*n/R], twiddles input r by
// w_{Ns*R}^{r*(j mod Ns)}, writes output r to y[(j/Ns)*Ns*R + (j mod Ns) + r*Ns]),
// but with n, R, Ns and the thread count known at compile time, so every index,
// division and loop bound folds to constants.  Loads and stores go through
// accessor objects, so a kernel can feed the first stage straight from global
// memory (or from its own computation) and take the last stage's outputs
// straight from registers.
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
  __host__ __device__ static constexpr int min_radix() {
    int m = R0;
    for (int i = 1; i < S; ++i) m = r(i) < m ? r(i) : m;
    return m;
  }
  static_assert(R0 * R1 * R2 * R3 == N_, "radices must multiply to N");
  // the reversed plan: the inverse transform that follows a forward one
  using Rev = typename std::conditional<
      S == 1, Spec<N_, R0>,
      typename std::conditional<
          S == 2, Spec<N_, R1, R0>,
          typename std::conditional<S == 3, Spec<N_, R2, R1, R0>, Spec<N_, R3, R2, R1, R0>>::type>::type>::type;
};

// Stage I of plan SP run by T threads over NC interleaved transforms
// (butterfly g = t + it*T of the stage maps to j = g / NC, c = g % NC).
template <class SP, int I, int T, int NC = 1>
struct StageC {
  static constexpr int N = SP::N;
  static constexpr int R = SP::r(I);
  static constexpr int NS = SP::ns(I);
  static constexpr int NB = N / R;
  static constexpr int UNIT = N / (NS * R);
  static constexpr int NCOL = NC;
  static constexpr int TOTAL = NB * NC;
  static constexpr int THREADS = T;
  static constexpr int IT = (TOTAL + T - 1) / T;
  static constexpr bool EXACT = (TOTAL % T) == 0;
};

template <class STG>
__device__ __forceinline__ bool stage_valid(int t, int it) {
  if constexpr (STG::EXACT) return true;
  else return t + it * STG::THREADS < STG::TOTAL;
}
template <class STG>
__device__ __forceinline__ int stage_j(int t, int it) {
  return (t + it * STG::THREADS) / STG::NCOL;
}
template <class STG>
__device__ __forceinline__ int stage_c(int t, int it) {
  return (t + it * STG::THREADS) % STG::NCOL;
}

// V[it][r] = ld(j + r*NB, c)
template <class STG, class LD>
__device__ __forceinline__ void stage_load(int t, const LD& ld, float2 (&V)[STG::IT][STG::R]) {
#pragma unroll
  for (int it = 0; it < STG::IT; ++it) {
    if (!stage_valid<STG>(t, it)) continue;
    const int j = stage_j<STG>(t, it), c = stage_c<STG>(t, it);
#pragma unroll
    for (int r = 0; r < STG::R; ++r) V[it][r] = ld(j + r * STG::NB, c);
  }
}

// twiddle the inputs and take the length-R DFT of every butterfly held
template <class STG, bool INV>
__device__ __forceinline__ void stage_compute(int t, const float2* __restrict__ tw, float2 (&V)[STG::IT][STG::R]) {
#pragma unroll
  for (int it = 0; it < STG::IT; ++it) {
    if (!stage_valid<STG>(t, it)) continue;
    if constexpr (STG::NS > 1) {
      const int k = stage_j<STG>(t, it) % STG::NS;
      twiddle_inputs<STG::R, INV>(V[it], k, STG::UNIT, tw);
    }
    Dft<STG::R, INV>::run(V[it]);
  }
}

// output index of element r of butterfly j
template <class STG>
__device__ __forceinline__ int stage_out(int j, int r) {
  if constexpr (STG::NS == 1) {
    return j * STG::R + r;
  } else {
    const int k = j % STG::NS;
    return (j - k) * STG::R + k + r * STG::NS;
  }
}

// st(out_index, c, value) for every output held
template <class STG, class ST>
__device__ __forceinline__ void stage_store(int t, const ST& st, float2 (&V)[STG::IT][STG::R]) {
#pragma unroll
  for (int it = 0; it < STG::IT; ++it) {
    if (!stage_valid<STG>(t, it)) continue;
    const int j = stage_j<STG>(t, it), c = stage_c<STG>(t, it);
#pragma unroll
    for (int r = 0; r < STG::R; ++r) st(stage_out<STG>(j, r), c, V[it][r]);
  }
}

// Out-of-place stage, one butterfly at a time (few registers): ld -> st.
template <class STG, bool INV, class LD, class ST>
__device__ __forceinline__ void stage_stream(int t, const float2* __restrict__ tw, const LD& ld, const ST& st) {
#pragma unroll
  for (int it = 0; it < STG::IT; ++it) {
    if (!stage_valid<STG>(t, it)) continue;
    const int j = stage_j<STG>(t, it), c = stage_c<STG>(t, it);
    float2 v[STG::R];
#pragma unroll
    for (int r = 0; r < STG::R; ++r) v[r] = ld(j + r * STG::NB, c);
    if constexpr (STG::NS > 1) twiddle_inputs<STG::R, INV>(v, j % STG::NS, STG::UNIT, tw);
    Dft<STG::R, INV>::run(v);
#pragma unroll
    for (int r = 0; r < STG::R; ++r) st(stage_out<STG>(j, r), c, v[r]);
  }
}

// ---------------------------------------------------------------- shared-memory accessors

// row layout: element i of the transform at p[i + (i >> 4)]
struct RowLd {
  const float2* p;
  __device__ __forceinline__ float2 operator()(int i, int) const { return p[rpad(i)]; }
};
struct RowSt {
  float2* p;
  __device__ __forceinline__ void operator()(int i, int, float2 v) const { p[rpad(i)] = v; }
};
// column layout: element i of column c at p[rpad(i*NC + c)]; the padding (one
// float2 per 16) spreads the stride-R*NC stores of the early stages over the banks
template <int NC>
struct ColLd {
  const float2* p;
  __device__ __forceinline__ float2 operator()(int i, int c) const { return p[rpad(i * NC + c)]; }
};
template <int NC>
struct ColSt {
  float2* p;
  __device__ __forceinline__ void operator()(int i, int c, float2 v) const { p[rpad(i * NC + c)] = v; }
};
__host__ __device__ constexpr int col_smem_len(int n, int nc) { return row_smem_len(n * nc); }

// Stages I0 .. I1-1 of SP, ping-pong between a and b (row layout), one
// barrier per stage.  Returns the buffer holding the result.
template <class SP, int I, int I1, int T, bool INV>
struct RowStagesPP {
  __device__ __forceinline__ static float2* run(float2* a, float2* b, int t, const float2* __restrict__ tw) {
    if constexpr (I < I1) {
      using STG = StageC<SP, I, T>;
      stage_stream<STG, INV>(t, tw, RowLd{a}, RowSt{b});
      __syncthreads();
      return RowStagesPP<SP, I + 1, I1, T, INV>::run(b, a, t, tw);
    } else {
      return a;
    }
  }
};

// Stages I .. I1-1 of SP in place (column layout): load all, barrier,
// transform and store, barrier.
template <class SP, int I, int I1, int T, int NC, bool INV>
struct ColStagesIP {
  __device__ __forceinline__ static void run(float2* p, int t, const float2* __restrict__ tw) {
    if constexpr (I < I1) {
      using STG = StageC<SP, I, T, NC>;
      float2 V[STG::IT][STG::R];
      stage_load<STG>(t, ColLd<NC>{p}, V);
      __syncthreads();
      stage_compute<STG, INV>(t, tw, V);
      stage_store<STG>(t, ColSt<NC>{p}, V);
      __syncthreads();
      ColStagesIP<SP, I + 1, I1, T, NC, INV>::run(p, t, tw);
    }
  }
};

}  // namespace prnu
