// search_fixed.cu -- compile-time-planned kernels of the grid search for the
// frame sizes of the workloads (256x256, 1280x720, 1920x1080, 3840x2160).
//
// Same arithmetic as the generic kernels in search.cu (Stockham stages,
// radix-R DFTs in registers, the same packed half spectrum), with the plan,
// the frame size and the thread count known at compile time, so that every
// address is a per-thread base plus a constant (fft_fixed.cuh), and with
// fewer shared-memory passes:
//   row_forward_body : stage 0 of the row FFT takes its inputs straight from
//                      the bilinear warp (no shared-memory fill);
//   col_body         : stage 0 loads the strip from global memory; the last
//                      forward stage, the spectrum product and the first
//                      inverse stage stay in registers (the inverse plan is
//                      the forward plan reversed, so every thread already
//                      holds its inputs); the last inverse stage stores to
//                      global memory; stages in between run in place; each
//                      thread works on a pair of adjacent columns;
//   row_inverse_body : stage 0 rebuilds the two rows' full spectrum straight
//                      from global memory; the last stage's outputs are
//                      reduced to the row statistics from registers.
// Each body runs either as its own wave kernel (one launch per phase over a
// wave of candidates) or inside k_persist, one launch that schedules all
// phases of all candidates of a call as tasks (see below).
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "fft_fixed.cuh"
#include "internal.h"
#include "search_common.cuh"
#include "search_fixed.h"
#include "tma.cuh"

namespace prnu {

namespace {

// Loads of spectra: L2-only (CG) inside the persistent kernel, whose blocks
// read what other blocks of the same launch wrote into reused slots; through
// the read-only path in the wave kernels, where the spectrum was written by an
// earlier launch.
template <bool CG>
__device__ __forceinline__ float2 ld_spec(const float2* p) {
  if constexpr (CG) return __ldcg(p);
  else return __ldg(p);
}
template <bool CG>
__device__ __forceinline__ float4 ld_spec4(const float4* p) {
  if constexpr (CG) return __ldcg(p);
  else return __ldg(p);
}

template <int W>
__host__ __device__ constexpr size_t row_fx_smem(int ppb) {
  return (size_t)ppb * row_len2(W) * sizeof(float2) + (size_t)ppb * 32 * sizeof(WarpRed);
}
__host__ __device__ constexpr size_t col_fx_smem(int H, int nc) { return (size_t)H * nc * sizeof(float2); }

// ---------------------------------------------------------------- row forward

// The 16 warped samples x = t + r*NB0 (r < 16) of output rows y0 and y0 + 1,
// packed as one complex row (row y0 real, row y0 + 1 imaginary).  CLAMP
// false is only taken when every sample point of the row pair lies in
// [-1, W] x [-1, H], where the clamp of bilinear_pad is the identity.
template <int DT, int W, int NB0, bool CLAMP>
__device__ __forceinline__ void warp_row16(const typename StoreT<DT>::type* __restrict__ fr, int H, const WorkItem& it,
                                           float dxj, float bx0, float by0, float bx1, float by1, float2 (&v)[16]) {
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const float dx = dxj + (float)(r * NB0);
    v[r].x = bilinear_pad<DT, W, CLAMP>(fr, H, fmaf(it.a11, dx, bx0), fmaf(it.a21, dx, by0));
    v[r].y = bilinear_pad<DT, W, CLAMP>(fr, H, fmaf(it.a11, dx, bx1), fmaf(it.a21, dx, by1));
  }
}

__device__ __forceinline__ bool in_box(float qx, float qy, int W, int H) {
  return qx >= -1.f && qx <= (float)W && qy >= -1.f && qy <= (float)H;
}

// Row pairs bx*PPB .. bx*PPB+PPB-1 of candidate `is` (item slot), spectrum
// written to workspace slot `ws`.  Block = PPB groups of T threads.
template <int DT, class SP, int T, int PPB>
__device__ __forceinline__ void row_forward_body(const PassArgs& a, int is, int ws, int bx, float2* smem, int tx) {
  constexpr int W = SP::N, Wh = W / 2, L = row_len2(W);
  using S0 = Stg<SP, 0>;
  static_assert(S0::R == 16 && SP::S >= 2 && SP::S <= 3, "row plans: radix 16 first, two or three stages");
  constexpr int NB0 = S0::NB;
  const int grp = tx / T, t = tx - grp * T;
  const int H = a.H;
  const int pair = bx * PPB + grp;
  float2* A = smem + (size_t)grp * L;   // the row pair's buffer; stages 1.. run in place
  const WorkItem it = item_of(a, is);
  size_t base;
  const void* Rf = frame_of(a, it.frame, &base);
  const auto* fr = reinterpret_cast<const typename StoreT<DT>::type*>(Rf) + base;
  const int y0 = 2 * pair;
  const float cx = 0.5f * (float)(W - 1), cy = 0.5f * (float)(H - 1);
  const float dy0 = (float)y0 - cy, dy1 = dy0 + 1.f;
  const float bx0 = fmaf(it.a12, dy0, cx), by0 = fmaf(it.a22, dy0, cy);
  const float bx1 = fmaf(it.a12, dy1, cx), by1 = fmaf(it.a22, dy1, cy);
  // The sample coordinates are monotone in x, so the ends of the two rows
  // bound them all (uniform over the thread group).
  const float dxl = -cx, dxr = (float)(W - 1) - cx;
  const bool inside = in_box(fmaf(it.a11, dxl, bx0), fmaf(it.a21, dxl, by0), W, H) &&
                      in_box(fmaf(it.a11, dxr, bx0), fmaf(it.a21, dxr, by0), W, H) &&
                      in_box(fmaf(it.a11, dxl, bx1), fmaf(it.a21, dxl, by1), W, H) &&
                      in_box(fmaf(it.a11, dxr, bx1), fmaf(it.a21, dxr, by1), W, H);
  if (t < NB0) {
    float2 v[16];
    const float dxj = (float)t - cx;
    if (inside) warp_row16<DT, W, NB0, false>(fr, H, it, dxj, bx0, by0, bx1, by1, v);
    else warp_row16<DT, W, NB0, true>(fr, H, it, dxj, bx0, by0, bx1, by1, v);
    Dft<16, false>::run(v);
    row_store16(A, t, v);
  }
  __syncthreads();
  float2* o0 = a.spec + ((size_t)ws * H + y0) * Wh;
  float2* o1 = o0 + Wh;
  using LS = Stg<SP, SP::S - 1>;
  constexpr bool kShflSplit = SP::S == 3 && LS::NB == T && T % 32 == 0 && LS::R % 2 == 0;
  if constexpr (kShflSplit) {
    // The last stage with butterflies j and Ns - j on partner lanes l and
    // l ^ 16 of one warp (j = 0 and Ns/2, their own mirrors, share lane pair
    // 0): output x = j + r*Ns has its mirror W - x at r' = R-1-r of butterfly
    // Ns - j, so the split of z = G_a + i G_b takes the mirror bins by shuffle
    // instead of a shared-memory round trip.
    row_stage_ip<SP, 1, T, false>(A, t);
    __syncthreads();
    constexpr int R = LS::R, NS = LS::NS, LB = NS / 16 * 18;
    const int p = (t >> 5) * 16 + (t & 15), h = (t >> 4) & 1;
    const int j = p == 0 ? (h ? NS / 2 : 0) : (h ? NS - p : p);
    float2 v[1][R];
    const float2* src = A + rp2(j);
#pragma unroll
    for (int r = 0; r < R; ++r) v[0][r] = src[r * LB];
    twiddle_tab<R, NS, false, 1>(v, j);
    Dft<R, false>::run(v[0]);
    float2 m[R / 2];
#pragma unroll
    for (int r = 0; r < R / 2; ++r) {
      m[r].x = __shfl_xor_sync(0xffffffffu, v[0][R - 1 - r].x, 16);
      m[r].y = __shfl_xor_sync(0xffffffffu, v[0][R - 1 - r].y, 16);
    }
#pragma unroll
    for (int r = 0; r < R / 2; ++r) {
      const int x = j + r * NS;   // < W/2
      const float2 zk = v[0][r];
      float2 P, Q;
      if (j == 0 && r == 0) {     // bin 0 packs (DC, Nyquist); the Nyquist bin W/2 is r = R/2 here
        const float2 zn = v[0][R / 2];
        P = make_float2(zk.x, zn.x);
        Q = make_float2(zk.y, zn.y);
      } else {
        const float2 zm = j == 0 ? v[0][R - r] : j == NS / 2 ? v[0][R - 1 - r] : m[r];
        P = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        Q = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
      }
      o0[x] = P;
      o1[x] = Q;
    }
    return;
  }
  const float2* res = A;
  row_stage_ip<SP, 1, T, false>(A, t);
  __syncthreads();
  if constexpr (SP::S == 3) {
    row_stage_ip<SP, 2, T, false>(A, t);
    __syncthreads();
  }
  // split z = G_a + i G_b into the two rows' half spectra (packed: bin 0
  // holds (DC, Nyquist))
  constexpr int MI = (Wh + T - 1) / T;
  const float2* rk = res + rp2(t);
  const float2* rm = res - t + 2 * ((-t) >> 4);   // + rp2(X) gives rp2(X - t) for X = 0 mod 16
#pragma unroll
  for (int m = 0; m < MI; ++m) {
    const int k = t + m * T;
    if (Wh % T != 0 && k >= Wh) break;
    const float2 zk = rk[m * (T / 16 * 18)];
    float2 P, Q;
    if (m == 0 && t == 0) {
      const float2 zn = res[rp2(Wh)];
      P = make_float2(zk.x, zn.x);
      Q = make_float2(zk.y, zn.y);
    } else {
      const float2 zm = rm[rp2(W - m * T)];
      P = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      Q = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
    }
    o0[k] = P;
    o1[k] = Q;
  }
}

// ---------------------------------------------------------------- column pass

// The fingerprint bins (i, col0) and (i, col0 + 1) for i = j + r*NS.
template <int R, int NS, int Wh>
__device__ __forceinline__ void load_fp_pair(const FpDesc& fp, int j, int col0, float2 (&s)[2][R]) {
  const size_t b = ((size_t)j * Wh + col0) / 2;
  if (fp.dtype == kF32) {
    const float4* p = reinterpret_cast<const float4*>(fp.spec) + b;
#pragma unroll
    for (int r = 0; r < R; ++r) split2(__ldg(p + (size_t)r * NS * (Wh / 2)), s[0][r], s[1][r]);
  } else {
    const float2* p = reinterpret_cast<const float2*>(fp.spec) + b;   // two __half2
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float2 u = __ldg(p + (size_t)r * NS * (Wh / 2));
      s[0][r] = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
      s[1][r] = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
    }
  }
}

// The product for the packed column 0 (DC + i*Nyquist columns of two real
// spectra in one complex column): F, Fm the frame bins i and H - i, S, Sm the
// fingerprint bins; unpack both, conj-multiply each real column's spectrum,
// repack.
__device__ __forceinline__ float2 packed_col0_product(float2 F, float2 Fm, float2 S, float2 Sm) {
  const float2 Aa = make_float2(0.5f * (F.x + Fm.x), 0.5f * (F.y - Fm.y));
  const float2 Bb = make_float2(0.5f * (F.y + Fm.y), 0.5f * (Fm.x - F.x));
  const float2 Ka = make_float2(0.5f * (S.x + Sm.x), 0.5f * (S.y - Sm.y));
  const float2 Kb = make_float2(0.5f * (S.y + Sm.y), 0.5f * (Sm.x - S.x));
  const float2 p1 = c_conj_mul(Aa, Ka), p2 = c_conj_mul(Bb, Kb);
  return make_float2(p1.x - p2.y, p1.y + p2.x);
}

// Rows per TMA box of an H-row strip of NC columns (float2): a divisor of H of
// at most 256 rows whose box size is a multiple of 128 bytes, so that every
// box lands 128-byte aligned in shared memory.
__host__ __device__ constexpr int tma_box_rows(int H, int NC, int esize = 8) {
  for (int br = 256; br >= 1; --br)
    if (H % br == 0 && (br * NC * esize) % 128 == 0) return br;
  return 0;
}
__host__ __device__ constexpr int fp_tmap_index(int NC) { return NC == 2 ? 0 : NC == 4 ? 1 : NC == 8 ? 2 : 3; }
__host__ __device__ constexpr size_t col_fx_smem_fpt(int H, int nc) { return (size_t)H * (nc + 1) * sizeof(float2); }
// bytes per fingerprint bin of the separate fingerprint region (MODE 3: FP32
// or FP16 bins; MODE 4: FP16 bins only)
__host__ __device__ constexpr int fp_region_bin(int mode) { return mode == 3 ? 8 : mode == 4 ? 4 : 0; }
__host__ __device__ constexpr size_t col_fx_smem_sep(int H, int nc, int mode) {
  return (size_t)H * nc * (sizeof(float2) + fp_region_bin(mode));
}
constexpr long long kTmaWaitPolls = 1ll << 20;   // polls of mbarrier.try_wait before giving up

// The column pass from the last forward stage on, for the strip of NC
// columns from c0 whose forward stages have run in the strip buffer sm (PART
// 2: which holds the last forward stage's outputs): the last forward stage,
// the product with the fingerprint fp, the inverse stages; the last inverse
// stage leaves the strip in sm (MODE >= 1) or in Z (MODE 0).  PART 1 stops
// after the last forward stage and leaves its outputs in sm, in natural
// order.  With MODE 2 the fingerprint strip comes by TMA into sm once every
// thread holds its inputs (fp_tma_ok: the caller allows it), completing the
// mbarrier bar (its completions so far: bar_uses, advanced here when the copy
// is made, the same on every thread); X0 is the packed column-0 scratch (H
// float2 that the fingerprint strip does not cover).  With MODE 3 and 4 the
// caller has already issued the fingerprint strip's copy into its own region
// after the strip (fp_tma_ok: it did), completing fbar once; X0 is then the
// strip buffer itself, free once every thread holds its inputs (PART 2 needs
// no X0: it multiplies as it loads).  hook() runs on every thread right after
// the barrier that follows the loads of the last forward stage (the strip
// buffer's old contents are then no longer needed).
// t = threadIdx.x.  Returns false if the fingerprint copy did not land in
// time (a.err raised).
template <class SP, int W, int NC, int T, int MODE, int PART, class Hook>
__device__ __forceinline__ bool col_tail(const PassArgs& a, const FpDesc& fp, int c0, float2* sm, float2* Z,
                                         uint64_t* bar, int& bar_uses, bool fp_tma_ok, float2* X0, Hook&& hook,
                                         int t, uint64_t* fbar = nullptr) {
  constexpr bool TMA = MODE >= 1, FPT = MODE >= 2 && PART != 1, FPSEP = MODE >= 3;
  constexpr int H = SP::N, Wh = W / 2;
  using IS = typename SP::Rev;
  using M = ColMap<NC, T>;
  constexpr int NP = M::NP, TJ = M::TJ;
  const int cp = t % NP, j0 = t / NP;
  const int col0 = c0 + 2 * cp;
  float4* sm4 = reinterpret_cast<float4*>(sm);
  // last forward stage -> spectrum product -> first inverse stage, in registers
  using FL = Stg<SP, SP::S - 1>;
  using I0 = Stg<IS, 0>;
  static_assert(I0::R == FL::R && I0::NB == FL::NB && FL::NB == FL::NS, "register hand-off needs the reversed plan");
  constexpr int IT = (FL::NB + TJ - 1) / TJ;
  float2 v[IT][2][FL::R];
  // The fingerprint strip comes by TMA (into the strip buffer with MODE 2,
  // into its own region with MODE 3/4), else by per-thread loads.
  const bool fp_tma = FPT && fp_tma_ok && fp.tmaps != nullptr && NC * (fp.dtype == kF32 ? 8 : 4) >= 16;
  char* const fpsm = reinterpret_cast<char*>(sm) + (FPSEP ? (size_t)H * NC * sizeof(float2) : 0);
  // fingerprint bin (i, col) of this strip
  auto fp_bin = [&](int i, int col) -> float2 {
    if (fp_tma) {
      if (fp.dtype == kF32) return reinterpret_cast<const float2*>(fpsm)[i * NC + (col - c0)];
      return __half22float2(reinterpret_cast<const __half2*>(fpsm)[i * NC + (col - c0)]);
    }
    return load_spec(fp.spec, fp.dtype, (size_t)i * Wh + col);
  };
  // the fingerprint bins (j + r*NS, col0) and (j + r*NS, col0 + 1) from the TMA'd strip
  auto fp_pair = [&](int j, int r, float2& s0, float2& s1) {
    if (fp.dtype == kF32) {
      split2(reinterpret_cast<const float4*>(fpsm)[(j + r * FL::NS) * NP + cp], s0, s1);
    } else {
      const float2 u = reinterpret_cast<const float2*>(fpsm)[(j + r * FL::NS) * NP + cp];   // two __half2
      s0 = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
      s1 = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
    }
  };
  if constexpr (PART == 2 && FPSEP) {
    // The strip holds the last forward stage's outputs in natural order and
    // the fingerprint strip has its own region: each bin is multiplied as it
    // is loaded, and column 0's mirror bins H - i are read from the strip.
    if (fp_tma) {
      const bool ok = mbar_wait_bounded(fbar, 0, kTmaWaitPolls);
      if (__syncthreads_or(!ok)) {
        if (t == 0) {
          if (a.err) atomicExch(a.err, 1);
          mbar_wait_bounded(fbar, 0, kTmaWaitPolls);
        }
        __syncthreads();
        return false;
      }
    }
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int j = j0 + it * TJ;
      if (FL::NB % TJ != 0 && j >= FL::NB) continue;
      const float4* src = sm4 + j * NP + cp;
      float2 sf[2][FL::R];
      if (!fp_tma) load_fp_pair<FL::R, FL::NS, Wh>(fp, j, col0, sf);
#pragma unroll
      for (int r = 0; r < FL::R; ++r) {
        float2 F0, F1, s0, s1;
        split2(src[r * FL::NB * NP], F0, F1);
        if (fp_tma) fp_pair(j, r, s0, s1);
        else {
          s0 = sf[0][r];
          s1 = sf[1][r];
        }
        if (col0 == 0) {
          const int i = j + r * FL::NS, im = i == 0 ? 0 : H - i;
          v[it][0][r] = packed_col0_product(F0, sm[im * NC], fp_bin(i, 0), fp_bin(im, 0));
        } else {
          v[it][0][r] = c_conj_mul(F0, s0);
        }
        v[it][1][r] = c_conj_mul(F1, s1);
      }
    }
    __syncthreads();   // every strip value read before the first inverse stage rewrites the strip
    hook();
  } else {
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int j = j0 + it * TJ;
    if (FL::NB % TJ != 0 && j >= FL::NB) continue;
    const float4* src = sm4 + j * NP + cp;
#pragma unroll
    for (int r = 0; r < FL::R; ++r) split2(src[r * FL::NB * NP], v[it][0][r], v[it][1][r]);
  }
  __syncthreads();
  hook();
  if constexpr (FPT && !FPSEP) {
    if (fp_tma && t == 0) {
      const CUtensorMap* fm = reinterpret_cast<const CUtensorMap*>(fp.tmaps) + fp_tmap_index(NC);
      const int es = fp.dtype == kF32 ? 8 : 4, fbr = tma_box_rows(H, NC, es);
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(fm))
                   : "memory");
      mbar_expect_tx(bar, H * NC * es);
#pragma unroll 1
      for (int b = 0; b < H / fbr; ++b)
        tma_load_2d(reinterpret_cast<char*>(sm) + (size_t)b * fbr * NC * es, fm, 2 * c0, b * fbr, bar);
    }
  }
  if constexpr (PART != 2) {   // PART 2: the strip held the outputs of this stage
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int j = j0 + it * TJ;
      if (FL::NB % TJ != 0 && j >= FL::NB) continue;
      twiddle_tab<FL::R, FL::NS, false, 2>(v[it], j);
      Dft<FL::R, false>::run(v[it][0]);
      Dft<FL::R, false>::run(v[it][1]);
    }
  }
  if constexpr (PART == 1) {
    // outputs i = j + r*NS go back where the stage took its inputs (NB == NS)
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int j = j0 + it * TJ;
      if (FL::NB % TJ != 0 && j >= FL::NB) continue;
      float4* dst = sm4 + j * NP + cp;
#pragma unroll
      for (int r = 0; r < FL::R; ++r) dst[r * FL::NS * NP] = join2(v[it][0][r], v[it][1][r]);
    }
    return true;
  }
  if constexpr (FPT) {
    if (fp_tma) {
      uint64_t* const wb = FPSEP ? fbar : bar;
      const int ph = FPSEP ? 0 : bar_uses & 1;
      if (!FPSEP) ++bar_uses;
      const bool ok = mbar_wait_bounded(wb, ph, kTmaWaitPolls);
      if (__syncthreads_or(!ok)) {
        if (t == 0) {
          if (a.err) atomicExch(a.err, 1);
          mbar_wait_bounded(wb, ph, kTmaWaitPolls);
        }
        __syncthreads();
        return false;
      }
    }
  }
  // thread holds bins i = j + r*NS of columns col0 and col0 + 1
  if (c0 == 0) {
    // packed column 0 (DC + i*Nyquist): the product needs bin H - i as well
    if (cp == 0) {
#pragma unroll
      for (int it = 0; it < IT; ++it) {
        const int j = j0 + it * TJ;
        if (FL::NB % TJ != 0 && j >= FL::NB) continue;
#pragma unroll
        for (int r = 0; r < FL::R; ++r) X0[j + r * FL::NS] = v[it][0][r];
      }
    }
    __syncthreads();
    if (cp == 0) {
#pragma unroll
      for (int it = 0; it < IT; ++it) {
        const int j = j0 + it * TJ;
        if (FL::NB % TJ != 0 && j >= FL::NB) continue;
#pragma unroll
        for (int r = 0; r < FL::R; ++r) {
          const int i = j + r * FL::NS;
          const int im = i == 0 ? 0 : H - i;
          v[it][0][r] = packed_col0_product(v[it][0][r], X0[im], fp_bin(i, 0), fp_bin(im, 0));
        }
      }
    }
    __syncthreads();
  }
  const bool col0_done = col0 == 0;
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int j = j0 + it * TJ;
    if (FL::NB % TJ != 0 && j >= FL::NB) continue;
    if (fp_tma) {
#pragma unroll
      for (int r = 0; r < FL::R; ++r) {
        float2 s0, s1;
        fp_pair(j, r, s0, s1);
        if (!col0_done) v[it][0][r] = c_conj_mul(v[it][0][r], s0);
        v[it][1][r] = c_conj_mul(v[it][1][r], s1);
      }
    } else {
      float2 sf[2][FL::R];
      load_fp_pair<FL::R, FL::NS, Wh>(fp, j, col0, sf);
#pragma unroll
      for (int r = 0; r < FL::R; ++r) {
        if (!col0_done) v[it][0][r] = c_conj_mul(v[it][0][r], sf[0][r]);
        v[it][1][r] = c_conj_mul(v[it][1][r], sf[1][r]);
      }
    }
  }
  if (!FPSEP && fp_tma) __syncthreads();   // every fingerprint bin read before the strip buffer is rewritten
  }
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int j = j0 + it * TJ;
    if (FL::NB % TJ != 0 && j >= FL::NB) continue;
    Dft<FL::R, true>::run(v[it][0]);
    Dft<FL::R, true>::run(v[it][1]);
    float4* dst = sm4 + j * FL::R * NP + cp;
#pragma unroll
    for (int r = 0; r < FL::R; ++r) dst[r * NP] = join2(v[it][0][r], v[it][1][r]);
  }
  __syncthreads();
  ColStages<IS, 1, IS::S - 1, T, NC, true>::run(sm4, t);

  {  // last inverse stage: shared memory -> global memory
    using G = Stg<IS, IS::S - 1>;
    static_assert(G::NB == G::NS, "last stage");
    constexpr int ITL = (G::NB + TJ - 1) / TJ;
#pragma unroll
    for (int it = 0; it < ITL; ++it) {
      const int j = j0 + it * TJ;
      if (G::NB % TJ != 0 && j >= G::NB) continue;
      float2 w[2][G::R];
      const float4* src = sm4 + j * NP + cp;
#pragma unroll
      for (int r = 0; r < G::R; ++r) split2(src[r * G::NB * NP], w[0][r], w[1][r]);
      twiddle_tab<G::R, G::NS, true, 2>(w, j);
      Dft<G::R, true>::run(w[0]);
      Dft<G::R, true>::run(w[1]);
      if constexpr (TMA) {
        // outputs j + r*Ns sit where this thread's inputs were: no barrier needed
        float4* dst = sm4 + j * NP + cp;
#pragma unroll
        for (int r = 0; r < G::R; ++r) dst[r * G::NS * NP] = join2(w[0][r], w[1][r]);
      } else {
        float4* dst = reinterpret_cast<float4*>(Z + (size_t)j * Wh + col0);
#pragma unroll
        for (int r = 0; r < G::R; ++r) dst[(size_t)r * G::NS * (Wh / 2)] = join2(w[0][r], w[1][r]);
      }
    }
  }
  return true;
}


// Columns bx*NC .. bx*NC+NC-1 of candidate `is` in workspace slot `ws`.
// MODE 0: every thread loads and stores its own elements.  MODE >= 1: the
// strip comes into shared memory by TMA tile copies through `map` (the
// workspace spectra as a [slots*H][W] float tensor) and leaves the same way.
// MODE 2: the fingerprint strip too comes by TMA, into the strip buffer once
// the last forward stage has taken its inputs (the packed column-0 scratch then
// sits after the strip).  MODE 3 and 4: the fingerprint strip comes by TMA
// into its own region after the strip buffer, copied from the start together
// with the strip (MODE 4 sizes the region for FP16 bins: FP32 fingerprints
// are then loaded per thread).  A TMA wait that runs out raises a.err and
// abandons the candidate.
// PART splits the pass for forward units (candidates that share a frame and
// a grid node): PART 1 runs the forward column FFT only and stores its
// output, in natural order, back to slot ws; PART 2 loads that output from
// slot src_ws, where each thread finds the values the last forward stage
// leaves in its registers, and runs the product and the inverse FFT into slot
// ws.  PART 1 then PART 2 compute bit for bit what PART 0 (the whole pass)
// computes.  PART 1 and 2 need TMA (MODE >= 1); PART 2 takes MODE 2.
template <class SP, int W, int NC, int T, bool CG = false, int MODE = 0, int PART = 0>
__device__ __forceinline__ void col_body(const PassArgs& a, int is, int ws, int bx, float2* sm,
                                         const CUtensorMap* map = nullptr, int src_ws = -1) {
  constexpr bool TMA = MODE >= 1, FPT = MODE >= 2 && PART != 1, FPSEP = MODE >= 3 && PART != 1;
  static_assert(PART == 0 || TMA, "the split column pass moves its strips by TMA");
  if (src_ws < 0) src_ws = ws;
  constexpr int H = SP::N, Wh = W / 2;
  using IS = typename SP::Rev;
  using M = ColMap<NC, T>;
  constexpr int NP = M::NP, TJ = M::TJ;
  static_assert(Wh % NC == 0, "strips tile the half spectrum");
  const int t = threadIdx.x;
  const int c0 = bx * NC;
  const int cp = t % NP, j0 = t / NP;
  const int col0 = c0 + 2 * cp;
  float2* Z = a.spec + (size_t)ws * H * Wh;
  float4* sm4 = reinterpret_cast<float4*>(sm);
  const WorkItem wi = item_of(a, is);
  const FpDesc fp = a.fps[wi.fp];

  constexpr int BR = tma_box_rows(H, NC);
  __shared__ uint64_t s_bar, s_fbar;
  // MODE 3/4: the fingerprint strip's copy goes out with the strip's (a
  // region sized for its bins, boxes of at least 16 bytes)
  const int fes = fp.dtype == kF32 ? 8 : 4;
  const bool fp_sep = FPSEP && fp.tmaps != nullptr && fes <= fp_region_bin(MODE) && NC * fes >= 16;
  if constexpr (TMA) {
    static_assert(BR > 0, "no TMA box for this strip");
    static_assert(!FPSEP || (H * NC * sizeof(float2)) % 128 == 0, "the fingerprint region starts 128-byte aligned");
    if (t == 0) {
      mbar_init(&s_bar, 1);
      if (FPSEP) mbar_init(&s_fbar, 1);
      fence_mbar_init();
    }
    __syncthreads();
    if (t == 0) {
      mbar_expect_tx(&s_bar, H * NC * 8 + (a.stall ? 16 : 0));   // the test hook waits for bytes that never come
#pragma unroll 1
      for (int b = 0; b < H / BR; ++b) tma_load_2d(sm + b * BR * NC, map, 2 * c0, src_ws * H + b * BR, &s_bar);
      if (fp_sep) {
        const CUtensorMap* fm = reinterpret_cast<const CUtensorMap*>(fp.tmaps) + fp_tmap_index(NC);
        const int fbr = tma_box_rows(H, NC, fes);
        char* dst = reinterpret_cast<char*>(sm) + (size_t)H * NC * sizeof(float2);
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(fm))
                     : "memory");
        mbar_expect_tx(&s_fbar, H * NC * fes);
#pragma unroll 1
        for (int b = 0; b < H / fbr; ++b) tma_load_2d(dst + (size_t)b * fbr * NC * fes, fm, 2 * c0, b * fbr, &s_fbar);
      }
    }
    const bool ok = mbar_wait_bounded(&s_bar, 0, kTmaWaitPolls);
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        if (a.err) atomicExch(a.err, 1);
        mbar_wait_bounded(&s_bar, 0, kTmaWaitPolls);   // let the copies land before the block leaves
        if (fp_sep) mbar_wait_bounded(&s_fbar, 0, kTmaWaitPolls);
      }
      __syncthreads();
      return;
    }
    if constexpr (PART != 2) ColStages<SP, 0, SP::S - 1, T, NC, false>::run(sm4, t);
  } else {  // forward stage 0 from global memory
    using G = Stg<SP, 0>;
    constexpr int IT = (G::NB + TJ - 1) / TJ;
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int j = j0 + it * TJ;
      if (G::NB % TJ != 0 && j >= G::NB) continue;
      float2 v[2][G::R];
      const float4* src = reinterpret_cast<const float4*>(Z + (size_t)j * Wh + col0);
#pragma unroll
      for (int r = 0; r < G::R; ++r) split2(ld_spec4<CG>(src + (size_t)r * G::NB * (Wh / 2)), v[0][r], v[1][r]);
      Dft<G::R, false>::run(v[0]);
      Dft<G::R, false>::run(v[1]);
      float4* dst = sm4 + j * G::R * NP + cp;
#pragma unroll
      for (int r = 0; r < G::R; ++r) dst[r * NP] = join2(v[0][r], v[1][r]);
    }
    __syncthreads();
    ColStages<SP, 1, SP::S - 1, T, NC, false>::run(sm4, t);
  }

  // the rest of the pass (PART 1 leaves its outputs in the strip buffer)
  float2* X0 = FPT && !FPSEP ? sm + H * NC : sm;   // with MODE 2 the strip buffer holds the fingerprint
  int bar_uses = 1;                                  // s_bar completed once (the strip)
  if (!col_tail<SP, W, NC, T, MODE, PART>(a, fp, c0, sm, Z, &s_bar, bar_uses, FPSEP ? fp_sep : true, X0, [] {}, t,
                                          &s_fbar))
    return;
  if constexpr (TMA) {
    fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
#pragma unroll 1
      for (int b = 0; b < H / BR; ++b) tma_store_2d(map, 2 * c0, ws * H + b * BR, sm + b * BR * NC);
      bulk_commit();
      if constexpr (CG) bulk_wait_all();
      else bulk_wait_read();
    }
  }
}

// ---------------------------------------------------------------- row inverse + statistics

// Inverse row FFT of z = G_a + i G_b, the full spectrum of the packed rows
// pa and pb (W/2 bins each), by the T threads of one group (thread t) with
// buffers A and B (row layout).  Afterwards thread t < n/R_last holds the
// outputs x = t + r*Ns_last of the last stage in v (v.x row a, v.y row b).
// Holds barriers: every thread of the block calls it.
template <class SP, int T, bool CG>
__device__ __forceinline__ void row_inverse_fft(const float2* pa, const float2* pb, float2* A, int t,
                                                float2 (&v)[RowLast<SP, T>::IT][RowLast<SP, T>::R]) {
  constexpr int W = SP::N, Wh = W / 2;
  using S0 = Stg<SP, 0>;
  static_assert(S0::R == 16 && SP::S >= 2 && SP::S <= 3, "row plans: radix 16 first, two or three stages");
  constexpr int NB0 = S0::NB;   // bins j + r*NB0: r < 8 below W/2, r >= 8 mirrored
  if (t < NB0) {
    float2 u[16];
    float2 a0 = make_float2(0.f, 0.f), b0 = a0;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const float2 A_ = ld_spec<CG>(pa + t + r * NB0), B_ = ld_spec<CG>(pb + t + r * NB0);
      if (r == 0) {
        a0 = A_;
        b0 = B_;
      }
      u[r] = make_float2(A_.x - B_.y, A_.y + B_.x);
    }
    const float2* ma = pa + (W - t);
    const float2* mb = pb + (W - t);
#pragma unroll
    for (int r = 8; r < 16; ++r) {
      float2 A_, B_;
      if (r == 8) {   // bin W/2 - t; for t = 0 the Nyquist bin, packed in bin 0
        const int k8 = t ? Wh - t : 0;
        A_ = ld_spec<CG>(pa + k8);
        B_ = ld_spec<CG>(pb + k8);
      } else {
        A_ = ld_spec<CG>(ma - r * NB0);
        B_ = ld_spec<CG>(mb - r * NB0);
      }
      u[r] = make_float2(A_.x + B_.y, B_.x - A_.y);
    }
    if (t == 0) {   // DC and Nyquist of both rows: (re, im) = (DC, Nyquist) in bin 0
      u[0] = make_float2(a0.x, b0.x);
      u[8] = make_float2(a0.y, b0.y);
    }
    Dft<16, true>::run(u);
    row_store16(A, t, u);
  }
  __syncthreads();
  if constexpr (SP::S == 3) {
    row_stage_ip<SP, 1, T, true>(A, t);
    __syncthreads();
  }
  row_stage_last<SP, T, true>(A, t, v);
}

template <class SP, int T, int PPB, bool CG = false>
__device__ __forceinline__ void row_inverse_body(const PassArgs& a, int ws, int bx, float2* smem, int tx) {
  constexpr int W = SP::N, Wh = W / 2, L = row_len2(W);
  using GL = RowLast<SP, T>;
  static_assert(PPB == 1 || T % 32 == 0, "row-pair groups must not share a warp (warp-level reductions)");
  const int grp = tx / T, t = tx - grp * T;
  const int H = a.H;
  const int pair = bx * PPB + grp;
  float2* A = smem + (size_t)grp * L;
  RowRed* red = reinterpret_cast<RowRed*>(smem + (size_t)PPB * L) + grp * 32;
  const float2* pa = a.spec + ((size_t)ws * H + 2 * pair) * Wh;
  float2 v[GL::IT][GL::R];
  row_inverse_fft<SP, T, CG>(pa, pa + Wh, A, t, v);
  // per thread: max, first arg-max and energy of each row over its outputs,
  // visited in increasing x (x = t + it*T + r*NS with t + it*T < NS), so a
  // strictly larger value is the only one that moves the arg-max: the first
  // maximum is kept without comparing indices
  float ma = -INFINITY, mb = -INFINITY;
  int ia = INT_MAX, ib = INT_MAX;
  float sa = 0.f, sb = 0.f;
#pragma unroll
  for (int r = 0; r < GL::R; ++r) {
#pragma unroll
    for (int it = 0; it < GL::IT; ++it) {
      if (!GL::valid(t, it)) continue;
      const int x = t + it * T + r * GL::NS;
      const float2 u = v[it][r];
      if (u.x > ma) {
        ma = u.x;
        ia = x;
      }
      if (u.y > mb) {
        mb = u.y;
        ib = x;
      }
      sa = fmaf(u.x, u.x, sa);
      sb = fmaf(u.y, u.y, sb);
    }
  }
  // across the warp: the max by an integer reduction of the order-preserving
  // key, then the least index among the lanes that hold it; energies by an
  // FP32 butterfly (warps are combined in double by row_stats_final)
  const int ka = __reduce_max_sync(0xffffffffu, float_key(ma));
  const int kb = __reduce_max_sync(0xffffffffu, float_key(mb));
  ia = __reduce_min_sync(0xffffffffu, float_key(ma) == ka ? ia : INT_MAX);
  ib = __reduce_min_sync(0xffffffffu, float_key(mb) == kb ? ib : INT_MAX);
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
  }
  if ((t & 31) == 0) red[t >> 5] = RowRed{key_float(ka), ia, key_float(kb), ib, sa, 0.f, sb, 0.f};
  __syncthreads();
  if (t == 0) row_stats_final(red, (T + 31) / 32, a.stats + (size_t)ws * H + 2 * pair);
}

// ---------------------------------------------------------------- wave kernels

// blockIdx.y = candidate slot, or with forward units the unit u, whose row
// spectrum goes to slot a.nitems + u
template <int DT, class SP, int T, int PPB>
__global__ void __launch_bounds__(T * PPB) k_row_forward_fx(PassArgs a) {
  extern __shared__ float4 smem4[];
  const bool units = a.units || a.share > 1;
  const int u = blockIdx.y;
  if (past_count(a, u, units ? 1 : 0)) return;
  row_forward_body<DT, SP, T, PPB>(a, units ? unit_first(a, u) : u, units ? a.nitems + u : u, blockIdx.x,
                                   reinterpret_cast<float2*>(smem4), threadIdx.x);
}

template <class SP, int W, int NC, int T, int MINB>
__global__ void __launch_bounds__(T, MINB) k_col_fx(PassArgs a) {
  extern __shared__ float4 smem4[];
  if (past_count(a, blockIdx.y, 0)) return;
  col_body<SP, W, NC, T>(a, blockIdx.y, blockIdx.y, blockIdx.x, reinterpret_cast<float2*>(smem4));
}

template <class SP, int W, int NC, int T, int MINB, int MODE>
__global__ void __launch_bounds__(T, MINB) k_col_tma_fx(PassArgs a, const __grid_constant__ CUtensorMap map) {
  extern __shared__ __align__(1024) float4 smem4t[];
  if (past_count(a, blockIdx.y, 0)) return;
  col_body<SP, W, NC, T, false, MODE>(a, blockIdx.y, blockIdx.y, blockIdx.x, reinterpret_cast<float2*>(smem4t),
                                      &map);
}

// Forward units (see col_body PART): the forward column FFT of unit
// blockIdx.y, in place in its slot a.nitems + u; then, per candidate slot
// blockIdx.y, the product with its fingerprint and the inverse FFT from its
// unit's slot into its own.
template <class SP, int W, int NC, int T, int MINB>
__global__ void __launch_bounds__(T, MINB) k_col_fwd_fx(PassArgs a, const __grid_constant__ CUtensorMap map) {
  extern __shared__ __align__(1024) float4 smem4f[];
  const int u = blockIdx.y;
  if (past_count(a, u, 1)) return;
  col_body<SP, W, NC, T, false, 1, 1>(a, unit_first(a, u), a.nitems + u, blockIdx.x,
                                      reinterpret_cast<float2*>(smem4f), &map);
}
template <class SP, int W, int NC, int T, int MINB, int MODE>
__global__ void __launch_bounds__(T, MINB) k_col_inv_fx(PassArgs a, const __grid_constant__ CUtensorMap map) {
  extern __shared__ __align__(1024) float4 smem4i[];
  const int s = blockIdx.y;
  if (past_count(a, s, 0)) return;
  col_body<SP, W, NC, T, false, MODE, 2>(a, s, s, blockIdx.x, reinterpret_cast<float2*>(smem4i), &map,
                                         a.nitems + unit_of_slot(a, s));
}

template <class SP, int T, int PPB>
__global__ void __launch_bounds__(T * PPB) k_row_inverse_fx(PassArgs a) {
  extern __shared__ float4 smem4[];
  if (past_count(a, blockIdx.y, 0)) return;
  row_inverse_body<SP, T, PPB>(a, blockIdx.y, blockIdx.x, reinterpret_cast<float2*>(smem4), threadIdx.x);
}
// the same with registers allocated for MINB resident blocks per SM (a
// separate kernel: an explicit bound of 1 changes the allocation of the
// unbounded one)
template <class SP, int T, int PPB, int MINB>
__global__ void __launch_bounds__(T * PPB, MINB) k_row_inverse_mb(PassArgs a) {
  extern __shared__ float4 smem4[];
  if (past_count(a, blockIdx.y, 0)) return;
  row_inverse_body<SP, T, PPB>(a, blockIdx.y, blockIdx.x, reinterpret_cast<float2*>(smem4), threadIdx.x);
}

// ---------------------------------------------------------------- persistent kernel

// Task bodies, inlined into k_persist.  The kernel hands them a thread index
// that the compiler cannot prove loop-invariant (see k_persist), so the
// per-thread index arithmetic of each task is computed inside its own branch
// instead of being hoisted out of the task loop, where the three tasks'
// values would all stay live at once.
template <int DT, class SP, int T, int PPB>
__device__ __forceinline__ void row_forward_task(const PassArgs& a, int is, int ws, int bx, float2* smem, int tx) {
  row_forward_body<DT, SP, T, PPB>(a, is, ws, bx, smem, tx);
}
template <class SP, int W, int NC, int T>
__device__ __forceinline__ void col_task(const PassArgs& a, int is, int ws, int bx, float2* smem) {
  col_body<SP, W, NC, T, true>(a, is, ws, bx, smem);
}
template <class SP, int T, int PPB>
__device__ __forceinline__ void row_inverse_task(const PassArgs& a, int ws, int bx, float2* smem, int tx) {
  row_inverse_body<SP, T, PPB, true>(a, ws, bx, smem, tx);
}

// finalize_body with the window's rows recomputed by the compile-time-planned
// inverse row FFT (one row pair per thread group, PPB pairs per round).
template <class SP, int T, int PPB>
__device__ __forceinline__ void finalize_task(const PassArgs& a, int is, int ws, float2* smem, int tx) {
  constexpr int W = SP::N, Wh = W / 2, L = row_len2(W), TB = T * PPB;
  using SL = RowLast<SP, T>;
  __shared__ int s_py, s_px, s_np;
  __shared__ float s_peak;
  __shared__ int s_pairs[2 * kHalfWindow + 1];
  const int t = tx, grp = t / T, tg = t - grp * T;
  const int H = a.H;
  const WorkItem it = item_of(a, is);
  const RowStat* st = a.stats + (size_t)ws * H;
  const float2* Z = a.spec + (size_t)ws * H * Wh;
  WarpRed* red = reinterpret_cast<WarpRed*>(smem + (size_t)PPB * L);
  constexpr int NW = TB / 32;
  const int w = t >> 5;

  float bv = -INFINITY;
  int bi = INT_MAX;
  for (int y = t; y < H; y += TB) {
    const RowStat r = ld_l2(st + y);
    better_f(bv, bi, r.max, y * W + r.arg);
  }
  warp_maxarg(bv, bi);
  if ((t & 31) == 0) {
    red[w].ma = bv;
    red[w].ia = bi;
  }
  __syncthreads();
  if (t == 0) {
    for (int k = 1; k < NW; ++k) better_f(bv, bi, red[k].ma, red[k].ia);
    if (bi == INT_MAX) bi = 0;
    s_peak = bv;
    s_py = bi / W;
    s_px = bi - (bi / W) * W;
    int np = 0, prev = -1;
    for (int d = -kHalfWindow; d <= kHalfWindow; ++d) {
      const int p = ((s_py + d + H) % H) >> 1;
      if (p != prev) s_pairs[np++] = p;
      prev = p;
    }
    s_np = np;
  }
  __syncthreads();
  const int py = s_py, px = s_px, np = s_np;
  double e = 0.0;
  for (int y = t; y < H; y += TB)
    if (cdist(y, py, H) > kHalfWindow) e += ld_l2(st + y).sumsq;
  for (int r0 = 0; r0 < np; r0 += PPB) {
    const int k = r0 + grp;
    const bool act = k < np;
    const int p = act ? s_pairs[k] : 0;
    float2* A = smem + (size_t)grp * L;
    const float2* pa = Z + (size_t)(2 * p) * Wh;
    float2 V[SL::IT][SL::R];
    row_inverse_fft<SP, T, true>(pa, pa + Wh, A, tg, V);
    if (act) {
#pragma unroll
      for (int it = 0; it < SL::IT; ++it) {
        if (!SL::valid(tg, it)) break;
#pragma unroll
        for (int r = 0; r < SL::R; ++r) {
          const int x = tg + it * T + r * SL::NS;
          if (cdist(x, px, W) <= kHalfWindow) continue;
          if (cdist(2 * p, py, H) <= kHalfWindow) e += (double)V[it][r].x * V[it][r].x;
          if (cdist(2 * p + 1, py, H) <= kHalfWindow) e += (double)V[it][r].y * V[it][r].y;
        }
      }
    }
    __syncthreads();
  }
  e = warp_sum(e);
  if ((t & 31) == 0) red[w].sa = e;
  __syncthreads();
  if (t == 0) {
    double etot = red[0].sa;
    for (int k = 1; k < NW; ++k) etot += red[k].sa;
    const double E = etot / ((double)H * (double)W - (double)kWindowCount);
    const double pk = (double)s_peak;
    double pce;
    if (E > 0.0) pce = (pk < 0 ? -1.0 : 1.0) * pk * pk / E;
    else pce = pk == 0.0 ? 0.0 : (pk < 0 ? -INFINITY : INFINITY);
    const FpDesc fp = a.fps[it.fp];
    double pv = pk / ((double)H * (double)W) * (double)(*fp.inv_scale);
    if (a.scale) pv /= (double)a.scale[it.frame];
    CandResult res;
    res.pce = pce;
    res.peak = (float)pv;
    res.py = py;
    res.px = px;
    res.cand = it.cand;
    res.group = it.group;
    res.pad = 0;
    *result_of(a, is) = res;
  }
}
// One block per candidate of the wave: finalize_task with PPB row pairs of the
// window recomputed at a time.
template <class SP, int T, int PPB>
__global__ void __launch_bounds__(T * PPB) k_finalize_fx(PassArgs a) {
  if (past_count(a, blockIdx.x, 0)) return;
  extern __shared__ float4 smem4[];
  finalize_task<SP, T, PPB>(a, blockIdx.x, blockIdx.x, reinterpret_cast<float2*>(smem4), threadIdx.x);
}

//
// One launch runs every phase of every candidate of a call.  Blocks take
// tasks by an atomic ticket.  Ticket order is a skewed pipeline: step s holds
// the row-forward tasks of candidate s, the column tasks of s-1, the
// row-inverse tasks of s-2 and the finalisation of s-3, so each task depends
// only on tasks with smaller tickets, which running blocks hold: the kernel
// cannot deadlock, whatever number of blocks is resident.  A task waits
// (bounded, with back-off) for the per-candidate count of its inputs; on
// timeout it raises the error flag and gives up instead of hanging.  Spectra
// and row statistics live in S workspace slots used round-robin (candidate g
// in slot g % S), so only about four candidates' spectra are in flight and
// they stay in L2; a row-forward task also waits for the finalisation of
// candidate g - S, the previous user of its slot.

constexpr long long kSpinLimit = 1ll << 23;   // ~2 s with the back-off below

__device__ __forceinline__ bool wait_count(const int* c, int need, int* err) {
  for (long long it = 0; it < kSpinLimit; ++it) {
    if (*(volatile const int*)c >= need) {
      __threadfence();
      return true;
    }
    if (*(volatile int*)err) return false;
    __nanosleep(it < 32 ? 64 : 256);
  }
  atomicExch(err, 1);
  return false;
}

template <int DT, class RS, int RT, int PPB, class CS, int NC>
__global__ void __launch_bounds__(RT * PPB, RT * PPB <= 384 ? 2 : 1)
    k_persist(const __grid_constant__ PassArgs a, const __grid_constant__ PersistArgs p) {
  constexpr int TB = RT * PPB;
  extern __shared__ float2 smem[];
  __shared__ int s_tk[2], s_ok, s_zero;
  static_assert(RT * PPB >= 64, "warp 1 publishes completions");
  const int H = a.H, Wh = a.W / 2;
  const int NRF = (H / 2) / PPB;
  const int NCOL = (Wh + NC - 1) / NC;
  const int NRI = NRF;
  const int TPS = NRF + NCOL + NRI + 1;
  const int total = (p.G + 3) * TPS;
  if (threadIdx.x == 0) {
    s_tk[0] = atomicAdd(p.ticket, 1);
    s_zero = 0;
  }
  __syncthreads();
  for (int iter = 0;; ++iter) {
    const int tk = s_tk[iter & 1];
    if (tk >= total) break;
    // the next ticket is fetched now and used after this task: its latency
    // overlaps the task instead of stalling the block
    int nxt = 0;
    if (threadIdx.x == 0) nxt = atomicAdd(p.ticket, 1);
    const int step = tk / TPS, r = tk - (tk / TPS) * TPS;
    int type, g, idx;
    if (r < NRF) {
      type = 0; g = step; idx = r;
    } else if (r < NRF + NCOL) {
      type = 1; g = step - 1; idx = r - NRF;
    } else if (r < NRF + NCOL + NRI) {
      type = 2; g = step - 2; idx = r - NRF - NCOL;
    } else {
      type = 3; g = step - 3; idx = 0;
    }
    if (g >= 0 && g < p.G) {   // uniform over the block
      const int ws = g % p.S;
      if (threadIdx.x == 0) {
        const int* dep = nullptr;
        int need = 1;
        if (type == 0) {
          if (g >= p.S) dep = p.fin_done + (g - p.S);
        } else if (type == 1) {
          dep = p.rf_done + g;
          need = NRF;
        } else if (type == 2) {
          dep = p.col_done + g;
          need = NCOL;
        } else {
          dep = p.ri_done + g;
          need = NRI;
        }
        s_ok = dep ? wait_count(dep, need + a.stall, p.error) : 1;   // the test hook waits for one count too many
      }
      __syncthreads();
      const bool ok = s_ok;
      if (ok) {
        const int tx = threadIdx.x + *(volatile int*)&s_zero;   // == threadIdx.x
        if (type == 0) row_forward_task<DT, RS, RT, PPB>(a, g, ws, idx, smem, tx);
        else if (type == 1) col_task<CS, RS::N, NC, TB>(a, g, ws, idx, smem);
        else if (type == 2) row_inverse_task<RS, RT, PPB>(a, ws, idx, smem, tx);
        else finalize_task<RS, RT, PPB>(a, g, ws, smem, tx);
      }
      __syncthreads();
      // completion is published by warp 1, so that warp 0 can go on to the
      // next ticket's dependency while the fence drains
      if (threadIdx.x == 32 && ok) {
        __threadfence();
        int* c = type == 0 ? p.rf_done : type == 1 ? p.col_done : type == 2 ? p.ri_done : p.fin_done;
        atomicAdd(c + g, 1);
      }
    }
    if (threadIdx.x == 0) s_tk[(iter + 1) & 1] = nxt;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- registry

template <class K>
void allow(K k) {
  allow_max_dynamic_smem(k);
}

// row pairs of the 11-row window recomputed at once by the finalisation
constexpr int kFinPairs = 3;

// RT threads per row pair in the row forward kernel, RTI in the row inverse
// (and in the finalisation)
template <class RS, int RT, class CS, int RTI = RT>
struct ShapeDef {
  static constexpr int W = RS::N, H = CS::N;
  // NC columns per block, CT threads, at least MINB resident blocks per SM
  // MODE: 0 plain loads and stores, 1 strip by TMA, 2 strip and fingerprint by TMA
  static FixedCol col_entry(void* fn, int nc, int ct, size_t smem, int mode) {
    allow_max_dynamic_smem(fn);
    FixedCol c{nc, ct, smem, fn, mode != 0, tma_box_rows(H, nc), mode};
    return c;
  }
  static constexpr size_t col_smem(int nc, int mode) {
    return mode >= 3 ? col_fx_smem_sep(H, nc, mode) : mode == 2 ? col_fx_smem_fpt(H, nc) : col_fx_smem(H, nc);
  }
  template <int NC, int CT, int MINB, int MODE>
  static FixedCol col() {
    void* fn = MODE ? (void*)k_col_tma_fx<CS, W, NC, CT, MINB, MODE> : (void*)k_col_fx<CS, W, NC, CT, MINB>;
    return col_entry(fn, NC, CT, col_smem(NC, MODE), MODE);
  }
  // the split column pass of forward units (NC columns, CT threads, MINB blocks)
  template <int NC, int CT, int MINB>
  static FixedCol col_fwd() {
    return col_entry((void*)k_col_fwd_fx<CS, W, NC, CT, MINB>, NC, CT, col_fx_smem(H, NC), 1);
  }
  template <int NC, int CT, int MINB, int MODE = 2>
  static FixedCol col_inv() {
    return col_entry((void*)k_col_inv_fx<CS, W, NC, CT, MINB, MODE>, NC, CT, col_smem(NC, MODE), MODE);
  }
  // RIMB: resident row-inverse blocks per SM to allocate registers for (0: no bound)
  template <int PPB, int RIMB = 0>
  static FixedRow row() {
    FixedRow r{};
    r.ppb = PPB;
    r.threads = RT;
    r.threads_inv = RTI;
    r.smem = row_fx_smem<W>(PPB);
    r.fwd[kF32] = (void*)k_row_forward_fx<kF32, RS, RT, PPB>;
    r.fwd[kF16] = (void*)k_row_forward_fx<kF16, RS, RT, PPB>;
    r.fwd[kBF16] = (void*)k_row_forward_fx<kBF16, RS, RT, PPB>;
    r.fwd[kF16P] = (void*)k_row_forward_fx<kF16P, RS, RT, PPB>;
    r.fwd[kBF16P] = (void*)k_row_forward_fx<kBF16P, RS, RT, PPB>;
    if constexpr (RIMB > 0) r.inv = (void*)k_row_inverse_mb<RS, RTI, PPB, RIMB>;
    else r.inv = (void*)k_row_inverse_fx<RS, RTI, PPB>;
    r.fin = (void*)k_finalize_fx<RS, RTI, kFinPairs>;
    r.fin_threads = RTI * kFinPairs;
    r.fin_smem = row_fx_smem<W>(kFinPairs);
    allow(k_finalize_fx<RS, RTI, kFinPairs>);
    allow(k_row_forward_fx<kF32, RS, RT, PPB>);
    allow(k_row_forward_fx<kF16, RS, RT, PPB>);
    allow(k_row_forward_fx<kBF16, RS, RT, PPB>);
    allow(k_row_forward_fx<kF16P, RS, RT, PPB>);
    allow(k_row_forward_fx<kBF16P, RS, RT, PPB>);
    allow_max_dynamic_smem(r.inv);
    return r;
  }
  // PRT threads per row pair (PRT * PPB per block, also the column task's
  // threads): chosen so that every stage holds one butterfly per thread
  template <int PRT, int PPB, int NC>
  static FixedPersist persist() {
    FixedPersist f{};
    f.ppb = PPB;
    f.nc = NC;
    f.threads = PRT * PPB;
    const size_t rs = row_fx_smem<W>(PPB);
    const size_t cs = col_fx_smem(H, NC);
    const size_t fs = row_fx_smem<W>(PPB);
    f.smem = std::max(rs, std::max(cs, fs));
    f.fn[kF32] = (void*)k_persist<kF32, RS, PRT, PPB, CS, NC>;
    f.fn[kF16] = (void*)k_persist<kF16, RS, PRT, PPB, CS, NC>;
    f.fn[kBF16] = (void*)k_persist<kBF16, RS, PRT, PPB, CS, NC>;
    for (int d = 0; d < 3; ++d) {
      allow_max_dynamic_smem(f.fn[d]);
      int nb = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f.fn[d], f.threads, f.smem);
      f.blocks_per_sm[d] = std::max(1, nb);
    }
    return f;
  }
  // split: the forward half, the inverse half (mode 2) and, optionally, the
  // inverse half with the fingerprint strip in its own region (mode 3/4) and
  // the one for FP16 fingerprints only (mode 4, more blocks per SM)
  static FixedShape make(std::vector<FixedRow> rows, std::vector<FixedCol> cols, std::vector<FixedCol> split,
                         FixedPersist ps) {
    FixedShape s{};
    s.W = W;
    s.H = H;
    s.rows = std::move(rows);
    s.cols = std::move(cols);
    s.col_fwd = split.at(0);
    s.col_inv = split.at(1);
    if (split.size() > 2) s.col_inv_sep = split[2];
    if (split.size() > 3) s.col_inv_h = split[3];
    s.persist = ps;
    return s;
  }
};

std::vector<FixedShape> build_registry() {
  std::vector<FixedShape> v;
  {
    using D = ShapeDef<Spec<1920, 16, 12, 10>, 192, Spec<1080, 9, 12, 10>, 160>;
    v.push_back(D::make({D::row<2>(), D::row<1, 8>()},
                        {D::col<4, 240, 3, 3>(), D::col<4, 240, 3, 2>(), D::col<4, 240, 3, 1>(),
                         D::col<4, 240, 3, 0>(), D::col<8, 480, 1, 1>()},
                        {D::col_fwd<4, 240, 3>(), D::col_inv<4, 240, 3>(), D::col_inv<4, 240, 3, 3>(),
                         D::col_inv<4, 240, 4, 4>()},
                        D::persist<192, 2, 4>()));
  }
  {
    using D = ShapeDef<Spec<1280, 16, 10, 8>, 160, Spec<720, 9, 10, 8>>;
    v.push_back(D::make({D::row<2>(), D::row<1>()},
                        {D::col<8, 360, 2, 3>(), D::col<8, 360, 2, 1>(), D::col<8, 360, 2, 2>(),
                         D::col<8, 360, 2, 0>(), D::col<4, 180, 4, 2>(), D::col<8, 360, 3, 4>()},
                        {D::col_fwd<4, 180, 4>(), D::col_inv<4, 180, 4>(), D::col_inv<4, 180, 4, 3>(),
                         D::col_inv<4, 180, 5, 4>()},
                        D::persist<160, 2, 4>()));
  }
  {
    using D = ShapeDef<Spec<3840, 16, 16, 15>, 256, Spec<2160, 15, 12, 12>>;
    v.push_back(D::make({D::row<2>(), D::row<1, 5>()},
                        {D::col<4, 360, 2, 4>(), D::col<4, 360, 2, 2>(), D::col<4, 360, 2, 1>(),
                         D::col<4, 360, 2, 0>()},
                        {D::col_fwd<4, 360, 2>(), D::col_inv<4, 360, 2>(), D::col_inv<4, 360, 2, 4>()},
                        D::persist<256, 2, 4>()));
  }
  {
    using D = ShapeDef<Spec<256, 16, 16>, 32, Spec<256, 16, 16>>;
    v.push_back(D::make({D::row<4>(), D::row<2>()},
                        {D::col<16, 128, 4, 2>(), D::col<16, 128, 4, 0>(), D::col<16, 128, 4, 3>()},
                        {D::col_fwd<16, 128, 4>(), D::col_inv<16, 128, 4>(), D::col_inv<16, 128, 4, 3>()},
                        D::persist<32, 8, 16>()));
  }
  cudaGetLastError();
  return v;
}

}  // namespace

const FixedShape* find_fixed(int H, int W) {
  static std::once_flag once;
  static std::vector<FixedShape> reg;
  std::call_once(once, [] { reg = build_registry(); });
  for (auto& s : reg)
    if (s.H == H && s.W == W) return &s;
  return nullptr;
}

bool fixed_supports(const FixedShape& fs, int H, int ppb) {
  const FixedRow& r = fs.row_for(ppb);
  return (H / 2) % r.ppb == 0;
}

namespace {

// cuTensorMapEncodeTiled from the driver, looked up once (nullptr if absent)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

// The workspace spectra [rows][W/2] float2 as a [rows][W] float tensor with
// boxes of br rows x 2*nc floats (nc complex columns).
bool encode_spec_map(CUtensorMap* m, const float2* base, int W, long long rows, int nc, int br) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || br <= 0) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)W * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)(2 * nc), (cuuint32_t)br};
  const cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

static_assert(4 * sizeof(CUtensorMap) == kFpTmapBytes, "four 128-byte descriptors per fingerprint");

bool encode_fp_tmaps(const void* spec, int dtype, int H, int W, void* out) {
  if (!find_fixed(H, W)) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const int es = dtype == kF32 ? 8 : 4;   // bytes per complex bin
  const int ncs[4] = {2, 4, 8, 16};
  CUtensorMap* m = reinterpret_cast<CUtensorMap*>(out);
  for (int k = 0; k < 4; ++k) {
    const int br = tma_box_rows(H, ncs[k], es);
    if (ncs[k] * es < 16) {   // a box row narrower than 16 bytes: no descriptor (the kernel loads per thread)
      memset(&m[k], 0, sizeof(CUtensorMap));
      continue;
    }
    if (br <= 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)W * (es / 2)};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * ncs[k]), (cuuint32_t)br};
    const cuuint32_t el[2] = {1, 1};
    if (enc(&m[k], es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
            const_cast<void*>(spec), dims, strides, box, el, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

void launch_fixed_wave(const PassArgs& a, const FixedShape& fs, int col_variant, cudaStream_t s, LaunchCounter& lc) {
  // forward units (several candidates of one frame and node): the row pass
  // and the forward column FFT per unit, into slots a.nitems + u; the product
  // and the inverse column FFT per candidate
  const bool units = a.units != nullptr || a.share > 1;
  const int nunits = units ? a.nunits : a.nitems;
  int v = std::max(0, std::min(col_variant, (int)fs.cols.size() - 1));
  // a variant whose fingerprint region holds FP16 bins only (mode 4) steps
  // aside for FP32 fingerprints: the first variant that copies FP32 bins by TMA
  if (fs.cols[v].mode == 4 && a.fp_f32)
    for (int k = 0; k < (int)fs.cols.size(); ++k)
      if (fs.cols[k].mode == 2 || fs.cols[k].mode == 3) {
        v = k;
        break;
      }
  const FixedCol& fv = fs.cols[v];
  // forward units take the split pass (its inverse half in the variant's fingerprint mode)
  const bool sep = fv.mode >= 3 && fs.col_inv_sep.fn && (fs.col_inv_sep.mode == 3 || !a.fp_f32);
  const bool sep_h = fv.mode >= 3 && fs.col_inv_h.fn && !a.fp_f32;
  const FixedCol& fc = units ? (sep_h ? fs.col_inv_h : sep ? fs.col_inv_sep : fs.col_inv) : fv;
  const FixedRow& fr = fs.row_for(a.pairs_per_block);
  const int Wh = a.W / 2;
  void* args[] = {const_cast<PassArgs*>(&a)};
  alignas(64) CUtensorMap map;
  const long long rows = (long long)(a.nitems + (units ? nunits : 0)) * a.H;
  if (fc.tma && !encode_spec_map(&map, a.spec, a.W, rows, fc.nc, fc.br))
    throw Error{PRNU_ECUDA, "cannot describe the workspace spectra for TMA (cuTensorMapEncodeTiled)"};
  void* targs[] = {const_cast<PassArgs*>(&a), &map};
  {
    ProfScope ps(lc, kKindRowForward, s);
    dim3 g((a.H / 2) / fr.ppb, nunits), b(fr.threads * fr.ppb);
    PRNU_CUDA_TRY(cudaLaunchKernel(fr.fwd[a.rdtype], g, b, args, fr.smem, s));
  }
  auto col_grid = [&](const FixedCol& c, int n) { return dim3((Wh + c.nc - 1) / c.nc, n); };
  if (units) {   // the forward half, per unit (same strip shape as the inverse half: one tensor map)
    ProfScope ps(lc, kKindColumn, s);
    const FixedCol& ff = fs.col_fwd;
    PRNU_CUDA_TRY(cudaLaunchKernel(ff.fn, col_grid(ff, nunits), dim3(ff.threads), targs, ff.smem, s));
    lc.n += 1;
  }
  {
    ProfScope ps(lc, kKindColumn, s);
    PRNU_CUDA_TRY(cudaLaunchKernel(fc.fn, col_grid(fc, a.nitems), dim3(fc.threads), fc.tma ? targs : args, fc.smem,
                                   s));
  }
  {
    ProfScope ps(lc, kKindRowInverse, s);
    dim3 g((a.H / 2) / fr.ppb, a.nitems), b(fr.threads_inv * fr.ppb);
    PRNU_CUDA_TRY(cudaLaunchKernel(fr.inv, g, b, args, fr.smem, s));
  }
  {
    ProfScope ps(lc, kKindFinalize, s);
    PRNU_CUDA_TRY(cudaLaunchKernel(fr.fin, dim3(a.nitems), dim3(fr.fin_threads), args, fr.fin_smem, s));
  }
  lc.n += 4;
}

void launch_persistent(const PassArgs& a, const PersistArgs& p, const FixedShape& fs, int sm_count, cudaStream_t s,
                       LaunchCounter& lc) {
  const FixedPersist& f = fs.persist;
  void* args[] = {const_cast<PassArgs*>(&a), const_cast<PersistArgs*>(&p)};
  ProfScope ps(lc, kKindFused, s);
  const int grid = sm_count * f.blocks_per_sm[a.rdtype];
  PRNU_CUDA_TRY(cudaLaunchKernel(f.fn[a.rdtype], dim3(grid), dim3(f.threads), args, f.smem, s));
  lc.n += 1;
}

}  // namespace prnu

