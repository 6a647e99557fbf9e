// search_fixed.cu -- compile-time-planned kernels of the grid search for the
// frame sizes of the workloads (256x256, 1280x720, 1920x1080, 3840x2160).
//
// Same arithmetic as the generic kernels in search.cu (the same Stockham
// stages and radix-R DFTs, the same packed half spectrum), with the plan known
// at compile time and fewer shared-memory passes:
//   row_forward_body : stage 0 of the row FFT takes its inputs straight from
//                      the bilinear warp (no shared-memory fill);
//   col_body         : stage 0 loads the strip from global memory; the last
//                      forward stage, the spectrum product and the first
//                      inverse stage stay in registers (the inverse plan is
//                      the forward plan reversed, so every thread already
//                      holds its inputs); the last inverse stage stores to
//                      global memory; stages in between run in place;
//   row_inverse_body : stage 0 rebuilds the two rows' full spectrum straight
//                      from global memory; the last stage's outputs are
//                      reduced to the row statistics from registers.
// Each body runs either as its own wave kernel (one launch per phase over a
// wave of candidates) or inside k_persist, one launch that schedules all
// phases of all candidates of a call as tasks (see below).
#include <algorithm>

#include "fft_fixed.cuh"
#include "internal.h"
#include "search_common.cuh"
#include "search_fixed.h"

namespace prnu {

namespace {

// Loads of spectra: L2-only (CG) inside the persistent kernel, whose blocks
// read what other blocks of the same launch wrote into reused slots; plain
// (L1-cached) in the wave kernels, where the row inverse reads every packed
// element twice (for bins k and W - k).
template <bool CG>
__device__ __forceinline__ float2 ld_spec(const float2* p) {
  if constexpr (CG) return ld_l2(p);
  else return *p;
}

// full spectrum element i of z = G_a + i G_b from two packed rows
template <bool CG>
struct FullRowLd {
  const float2* pa;
  const float2* pb;
  int W, Wh;
  __device__ __forceinline__ float2 operator()(int i, int) const {
    if (i == 0) {
      const float2 A = ld_spec<CG>(pa), B = ld_spec<CG>(pb);
      return make_float2(A.x, B.x);
    }
    if (i == Wh) {
      const float2 A = ld_spec<CG>(pa), B = ld_spec<CG>(pb);
      return make_float2(A.y, B.y);
    }
    if (i < Wh) {
      const float2 A = ld_spec<CG>(pa + i), B = ld_spec<CG>(pb + i);
      return make_float2(A.x - B.y, A.y + B.x);
    }
    const int k = W - i;
    const float2 A = ld_spec<CG>(pa + k), B = ld_spec<CG>(pb + k);
    return make_float2(A.x + B.y, B.x - A.y);
  }
};

template <bool CG>
struct StripLd {
  const float2* Z;
  int Wh, c0;
  __device__ __forceinline__ float2 operator()(int i, int c) const {
    const int col = c0 + c;
    return col < Wh ? ld_spec<CG>(Z + (size_t)i * Wh + col) : make_float2(0.f, 0.f);
  }
};
struct StripSt {
  float2* Z;
  int Wh, c0;
  __device__ __forceinline__ void operator()(int i, int c, float2 v) const {
    const int col = c0 + c;
    if (col < Wh) Z[(size_t)i * Wh + col] = v;
  }
};

template <int W>
__host__ __device__ constexpr size_t row_fx_smem(int ppb) {
  return (size_t)ppb * 2 * row_smem_len(W) * sizeof(float2) + (size_t)ppb * 32 * sizeof(WarpRed);
}

// ---------------------------------------------------------------- row forward

// Row pairs bx*PPB .. bx*PPB+PPB-1 of candidate `is` (item slot), spectrum
// written to workspace slot `ws`.  Block = PPB groups of T threads.
template <int DT, class SP, int T, int PPB>
__device__ __forceinline__ void row_forward_body(const PassArgs& a, int is, int ws, int bx, float2* smem, int tx) {
  constexpr int W = SP::N, Wh = W / 2, L = row_smem_len(W);
  const int grp = tx / T, t = tx - grp * T;
  const int H = a.H;
  const int pair = bx * PPB + grp;
  float2* A = smem + (size_t)grp * 2 * L;
  float2* B = A + L;
  const float2* tw = a.tw + a.prow.tw_off;
  const WorkItem it = item_of(a, is);
  size_t base;
  const void* Rf = frame_of(a, it.frame, &base);
  const auto* fr = reinterpret_cast<const typename StoreT<DT>::type*>(Rf) + base;
  const int y0 = 2 * pair;
  const float cx = 0.5f * (float)(W - 1), cy = 0.5f * (float)(H - 1);
  const float dy0 = (float)y0 - cy, dy1 = dy0 + 1.f;
  const float bx0 = fmaf(it.a12, dy0, cx), by0 = fmaf(it.a22, dy0, cy);
  const float bx1 = fmaf(it.a12, dy1, cx), by1 = fmaf(it.a22, dy1, cy);
  using S0 = StageC<SP, 0, T>;
#pragma unroll
  for (int k = 0; k < S0::IT; ++k) {
    if (!stage_valid<S0>(t, k)) continue;
    const int j = t + k * T;
    float2 v[S0::R];
#pragma unroll
    for (int r = 0; r < S0::R; ++r) {
      const float dx = (float)(j + r * S0::NB) - cx;
      v[r].x = bilinear_pad<DT, W>(fr, H, fmaf(it.a11, dx, bx0), fmaf(it.a21, dx, by0));
      v[r].y = bilinear_pad<DT, W>(fr, H, fmaf(it.a11, dx, bx1), fmaf(it.a21, dx, by1));
    }
    Dft<S0::R, false>::run(v);
#pragma unroll
    for (int r = 0; r < S0::R; ++r) A[rpad(j * S0::R + r)] = v[r];
  }
  __syncthreads();
  const float2* res = RowStagesPP<SP, 1, SP::S, T, false>::run(A, B, t, tw);
  float2* o0 = a.spec + ((size_t)ws * H + y0) * Wh;
  float2* o1 = o0 + Wh;
  for (int k = t; k < Wh; k += T) {
    float2 P, Q;
    if (k == 0) {
      const float2 z0 = res[rpad(0)], zn = res[rpad(Wh)];
      P = make_float2(z0.x, zn.x);
      Q = make_float2(z0.y, zn.y);
    } else {
      const float2 zk = res[rpad(k)], zm = res[rpad(W - k)];
      P = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      Q = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
    }
    o0[k] = P;
    o1[k] = Q;
  }
}

// ---------------------------------------------------------------- column pass

// Columns bx*NC .. bx*NC+NC-1 of candidate `is` in workspace slot `ws`.
template <class SP, int NC, int T, bool CG = false, bool PF = true>
__device__ __forceinline__ void col_body(const PassArgs& a, int is, int ws, int bx, float2* sm, int tx) {
  constexpr int H = SP::N;
  using IS = typename SP::Rev;
  const int t = threadIdx.x;   // == tx; the builtin gives this body the faster schedule (measured)
  const int Wh = a.W >> 1;
  const int c0 = bx * NC;
  float2* Z = a.spec + (size_t)ws * H * Wh;
  const float2* tw = a.tw + a.pcol.tw_off;
  const WorkItem wi = item_of(a, is);
  const FpDesc fp = a.fps[wi.fp];
  using FL = StageC<SP, SP::S - 1, T, NC>;
  using I0 = StageC<IS, 0, T, NC>;

  // The fingerprint bins this thread multiplies after the last forward stage
  // are known now: load them first, so that their latency hides behind the
  // forward stages (when they fit in a few registers and PF allows it).
  constexpr bool kPrefetch = PF && FL::IT * FL::R <= 16;
  float2 Sp[kPrefetch ? FL::IT : 1][kPrefetch ? FL::R : 1];
  if constexpr (kPrefetch) {
#pragma unroll
    for (int k = 0; k < FL::IT; ++k) {
      if (!stage_valid<FL>(t, k)) continue;
      const int j = stage_j<FL>(t, k), col = c0 + stage_c<FL>(t, k);
#pragma unroll
      for (int r = 0; r < FL::R; ++r)
        Sp[k][r] = col < Wh ? load_spec(fp.spec, fp.dtype, (size_t)(j + r * FL::NS) * Wh + col)
                            : make_float2(0.f, 0.f);
    }
  }

  stage_stream<StageC<SP, 0, T, NC>, false>(t, tw, StripLd<CG>{Z, Wh, c0}, ColSt<NC>{sm});
  __syncthreads();
  ColStagesIP<SP, 1, SP::S - 1, T, NC, false>::run(sm, t, tw);
  static_assert(I0::R == FL::R && I0::NB == FL::NB && FL::NB == FL::NS, "register hand-off needs the reversed plan");
  float2 V[FL::IT][FL::R];
  stage_load<FL>(t, ColLd<NC>{sm}, V);
  __syncthreads();
  stage_compute<FL, false>(t, tw, V);
  // outputs of the last forward stage: row i = j + r*NS of column c
  if (c0 == 0) {
    // packed column 0 (DC + i*Nyquist): the product needs row H - i as well
#pragma unroll
    for (int k = 0; k < FL::IT; ++k) {
      if (!stage_valid<FL>(t, k) || stage_c<FL>(t, k) != 0) continue;
      const int j = stage_j<FL>(t, k);
#pragma unroll
      for (int r = 0; r < FL::R; ++r) sm[rpad((j + r * FL::NS) * NC)] = V[k][r];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < FL::IT; ++k) {
      if (!stage_valid<FL>(t, k) || stage_c<FL>(t, k) != 0) continue;
      const int j = stage_j<FL>(t, k);
#pragma unroll
      for (int r = 0; r < FL::R; ++r) {
        const int i = j + r * FL::NS;
        const int im = i == 0 ? 0 : H - i;
        const float2 F = V[k][r], Fm = sm[rpad(im * NC)];
        const float2 S = load_spec(fp.spec, fp.dtype, (size_t)i * Wh);
        const float2 Sm = load_spec(fp.spec, fp.dtype, (size_t)im * Wh);
        const float2 Aa = make_float2(0.5f * (F.x + Fm.x), 0.5f * (F.y - Fm.y));
        const float2 Bb = make_float2(0.5f * (F.y + Fm.y), 0.5f * (Fm.x - F.x));
        const float2 Ka = make_float2(0.5f * (S.x + Sm.x), 0.5f * (S.y - Sm.y));
        const float2 Kb = make_float2(0.5f * (S.y + Sm.y), 0.5f * (Sm.x - S.x));
        const float2 p1 = c_mul(c_conj(Aa), Ka), p2 = c_mul(c_conj(Bb), Kb);
        V[k][r] = make_float2(p1.x - p2.y, p1.y + p2.x);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < FL::IT; ++k) {
    if (!stage_valid<FL>(t, k)) continue;
    const int j = stage_j<FL>(t, k), col = c0 + stage_c<FL>(t, k);
    if (col == 0 || col >= Wh) continue;
#pragma unroll
    for (int r = 0; r < FL::R; ++r) {
      float2 S;
      if constexpr (kPrefetch) S = Sp[k][r];
      else S = load_spec(fp.spec, fp.dtype, (size_t)(j + r * FL::NS) * Wh + col);
      V[k][r] = c_mul(c_conj(V[k][r]), S);
    }
  }
  stage_compute<I0, true>(t, tw, V);
  stage_store<I0>(t, ColSt<NC>{sm}, V);
  __syncthreads();
  ColStagesIP<IS, 1, IS::S - 1, T, NC, true>::run(sm, t, tw);
  stage_stream<StageC<IS, IS::S - 1, T, NC>, true>(t, tw, ColLd<NC>{sm}, StripSt{Z, Wh, c0});
}

// ---------------------------------------------------------------- row inverse + statistics

template <class SP, int T, int PPB, bool CG = false>
__device__ __forceinline__ void row_inverse_body(const PassArgs& a, int ws, int bx, float2* smem, int tx) {
  constexpr int W = SP::N, Wh = W / 2, L = row_smem_len(W);
  const int grp = tx / T, t = tx - grp * T;
  const int H = a.H;
  const int pair = bx * PPB + grp;
  float2* A = smem + (size_t)grp * 2 * L;
  float2* B = A + L;
  RowRed* red = reinterpret_cast<RowRed*>(smem + (size_t)PPB * 2 * L) + grp * 32;
  const float2* tw = a.tw + a.prow.tw_off;
  const float2* pa = a.spec + ((size_t)ws * H + 2 * pair) * Wh;
  stage_stream<StageC<SP, 0, T>, true>(t, tw, FullRowLd<CG>{pa, pa + Wh, W, Wh}, RowSt{A});
  __syncthreads();
  const float2* res = RowStagesPP<SP, 1, SP::S - 1, T, true>::run(A, B, t, tw);
  using SL = StageC<SP, SP::S - 1, T>;
  static_assert(SL::NB == SL::NS, "last stage writes j + r*NS");
  static_assert(PPB == 1 || T % 32 == 0, "row-pair groups must not share a warp (warp-level reductions)");
  float2 V[SL::IT][SL::R];
  stage_load<SL>(t, RowLd{res}, V);
  stage_compute<SL, true>(t, tw, V);
  float ma = -INFINITY, mb = -INFINITY;
  int ia = INT_MAX, ib = INT_MAX;
  float sa = 0.f, sb = 0.f;
#pragma unroll
  for (int k = 0; k < SL::IT; ++k) {
    if (!stage_valid<SL>(t, k)) continue;
    const int j = stage_j<SL>(t, k);
#pragma unroll
    for (int r = 0; r < SL::R; ++r) {
      const int x = j + r * SL::NS;
      const float2 v = V[k][r];
      better_f(ma, ia, v.x, x);
      better_f(mb, ib, v.y, x);
      sa = fmaf(v.x, v.x, sa);
      sb = fmaf(v.y, v.y, sb);
    }
  }
  row_stats_warp(ma, ia, mb, ib, sa, sb, t, red);
  __syncthreads();
  if (t == 0) row_stats_final(red, (T + 31) / 32, a.stats + (size_t)ws * H + 2 * pair);
}

// ---------------------------------------------------------------- wave kernels

template <int DT, class SP, int T, int PPB>
__global__ void __launch_bounds__(T * PPB) k_row_forward_fx(PassArgs a) {
  extern __shared__ float2 smem[];
  row_forward_body<DT, SP, T, PPB>(a, blockIdx.y, blockIdx.y, blockIdx.x, smem, threadIdx.x);
}

template <class SP, int NC, int T>
__global__ void __launch_bounds__(T) k_col_fx(PassArgs a) {
  extern __shared__ float2 smem[];
  col_body<SP, NC, T>(a, blockIdx.y, blockIdx.y, blockIdx.x, smem, threadIdx.x);
}

template <class SP, int T, int PPB>
__global__ void __launch_bounds__(T * PPB) k_row_inverse_fx(PassArgs a) {
  extern __shared__ float2 smem[];
  row_inverse_body<SP, T, PPB>(a, blockIdx.y, blockIdx.x, smem, threadIdx.x);
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
template <class SP, int NC, int T>
__device__ __forceinline__ void col_task(const PassArgs& a, int is, int ws, int bx, float2* smem, int tx) {
  col_body<SP, NC, T, true, false>(a, is, ws, bx, smem, tx);   // no prefetch: registers are capped here
}
template <class SP, int T, int PPB>
__device__ __forceinline__ void row_inverse_task(const PassArgs& a, int ws, int bx, float2* smem, int tx) {
  row_inverse_body<SP, T, PPB, true>(a, ws, bx, smem, tx);
}

// finalize_body with the window's rows recomputed by the compile-time-planned
// inverse row FFT (one row pair per thread group, PPB pairs per round).
template <class SP, int T, int PPB>
__device__ __forceinline__ void finalize_task(const PassArgs& a, int is, int ws, float2* smem, int tx) {
  constexpr int W = SP::N, Wh = W / 2, L = row_smem_len(W), TB = T * PPB;
  __shared__ int s_py, s_px, s_np;
  __shared__ float s_peak;
  __shared__ int s_pairs[2 * kHalfWindow + 1];
  const int t = tx, grp = t / T, tg = t - grp * T;
  const int H = a.H;
  const WorkItem it = item_of(a, is);
  const RowStat* st = a.stats + (size_t)ws * H;
  const float2* Z = a.spec + (size_t)ws * H * Wh;
  const float2* tw = a.tw + a.prow.tw_off;
  WarpRed* red = reinterpret_cast<WarpRed*>(smem + (size_t)PPB * 2 * L);
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
  using SL = StageC<SP, SP::S - 1, T>;
  for (int r0 = 0; r0 < np; r0 += PPB) {
    const int k = r0 + grp;
    const bool act = k < np;
    const int p = act ? s_pairs[k] : 0;
    float2* A = smem + (size_t)grp * 2 * L;
    float2* B = A + L;
    const float2* pa = Z + (size_t)(2 * p) * Wh;
    stage_stream<StageC<SP, 0, T>, true>(tg, tw, FullRowLd<true>{pa, pa + Wh, W, Wh}, RowSt{A});
    __syncthreads();
    const float2* res = RowStagesPP<SP, 1, SP::S - 1, T, true>::run(A, B, tg, tw);
    float2 V[SL::IT][SL::R];
    stage_load<SL>(tg, RowLd{res}, V);
    stage_compute<SL, true>(tg, tw, V);
    if (act) {
#pragma unroll
      for (int kk = 0; kk < SL::IT; ++kk) {
        if (!stage_valid<SL>(tg, kk)) continue;
        const int j = stage_j<SL>(tg, kk);
#pragma unroll
        for (int r = 0; r < SL::R; ++r) {
          const int x = j + r * SL::NS;
          if (cdist(x, px, W) <= kHalfWindow) continue;
          if (cdist(2 * p, py, H) <= kHalfWindow) e += (double)V[kk][r].x * V[kk][r].x;
          if (cdist(2 * p + 1, py, H) <= kHalfWindow) e += (double)V[kk][r].y * V[kk][r].y;
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
__global__ void __launch_bounds__(RT * PPB, 2) k_persist(const __grid_constant__ PassArgs a, const __grid_constant__ PersistArgs p) {
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
        s_ok = dep ? wait_count(dep, need, p.error) : 1;
      }
      __syncthreads();
      const bool ok = s_ok;
      if (ok) {
        const int tx = threadIdx.x + *(volatile int*)&s_zero;   // == threadIdx.x
        if (type == 0) row_forward_task<DT, RS, RT, PPB>(a, g, ws, idx, smem, tx);
        else if (type == 1) col_task<CS, NC, TB>(a, g, ws, idx, smem, tx);
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

template <class RS, int RT, class CS>
struct ShapeDef {
  static constexpr int W = RS::N, H = CS::N;
  template <int NC, int CT>
  static FixedCol col() {
    allow(k_col_fx<CS, NC, CT>);
    return FixedCol{NC, CT, (size_t)col_smem_len(H, NC) * sizeof(float2), (void*)k_col_fx<CS, NC, CT>};
  }
  template <int PPB>
  static FixedRow row() {
    FixedRow r{};
    r.ppb = PPB;
    r.threads = RT;
    r.smem = row_fx_smem<W>(PPB);
    r.fwd[kF32] = (void*)k_row_forward_fx<kF32, RS, RT, PPB>;
    r.fwd[kF16] = (void*)k_row_forward_fx<kF16, RS, RT, PPB>;
    r.fwd[kBF16] = (void*)k_row_forward_fx<kBF16, RS, RT, PPB>;
    r.inv = (void*)k_row_inverse_fx<RS, RT, PPB>;
    allow(k_row_forward_fx<kF32, RS, RT, PPB>);
    allow(k_row_forward_fx<kF16, RS, RT, PPB>);
    allow(k_row_forward_fx<kBF16, RS, RT, PPB>);
    allow(k_row_inverse_fx<RS, RT, PPB>);
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
    const size_t cs = (size_t)col_smem_len(H, NC) * sizeof(float2);
    const size_t fs = (size_t)2 * row_smem_len(W) * sizeof(float2) + 32 * sizeof(WarpRed);
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
  static FixedShape make(std::vector<FixedRow> rows, std::vector<FixedCol> cols, FixedPersist ps) {
    FixedShape s{};
    s.W = W;
    s.H = H;
    s.rows = std::move(rows);
    s.cols = std::move(cols);
    s.persist = ps;
    return s;
  }
};

std::vector<FixedShape> build_registry() {
  std::vector<FixedShape> v;
  {
    using D = ShapeDef<Spec<1920, 16, 12, 10>, 192, Spec<1080, 12, 10, 9>>;
    v.push_back(D::make({D::row<2>(), D::row<1>()},
                        {D::col<4, 480>(), D::col<8, 480>(), D::col<8, 960>(), D::col<16, 960>()},
                        D::persist<192, 2, 8>()));
  }
  {
    using D = ShapeDef<Spec<1280, 16, 10, 8>, 160, Spec<720, 10, 9, 8>>;
    v.push_back(D::make({D::row<2>(), D::row<1>()}, {D::col<4, 384>(), D::col<8, 384>(), D::col<16, 736>()},
                        D::persist<192, 2, 4>()));
  }
  {
    using D = ShapeDef<Spec<3840, 16, 16, 15>, 256, Spec<2160, 15, 12, 12>>;
    v.push_back(D::make({D::row<2>(), D::row<1>()}, {D::col<4, 384>(), D::col<4, 736>(), D::col<8, 736>()},
                        D::persist<384, 1, 2>()));
  }
  {
    using D = ShapeDef<Spec<256, 16, 16>, 32, Spec<256, 16, 16>>;
    v.push_back(D::make({D::row<4>(), D::row<2>()}, {D::col<8, 128>(), D::col<16, 256>()}, D::persist<32, 8, 16>()));
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

void launch_fixed_wave(const PassArgs& a, const FixedShape& fs, int col_variant, cudaStream_t s, LaunchCounter& lc) {
  const FixedCol& fc = fs.cols[std::max(0, std::min(col_variant, (int)fs.cols.size() - 1))];
  const FixedRow& fr = fs.row_for(a.pairs_per_block);
  const int Wh = a.W / 2;
  void* args[] = {const_cast<PassArgs*>(&a)};
  {
    ProfScope ps(lc, kKindRowForward, s);
    dim3 g((a.H / 2) / fr.ppb, a.nitems), b(fr.threads * fr.ppb);
    PRNU_CUDA_TRY(cudaLaunchKernel(fr.fwd[a.rdtype], g, b, args, fr.smem, s));
  }
  {
    ProfScope ps(lc, kKindColumn, s);
    dim3 g((Wh + fc.nc - 1) / fc.nc, a.nitems), b(fc.threads);
    PRNU_CUDA_TRY(cudaLaunchKernel(fc.fn, g, b, args, fc.smem, s));
  }
  {
    ProfScope ps(lc, kKindRowInverse, s);
    dim3 g((a.H / 2) / fr.ppb, a.nitems), b(fr.threads * fr.ppb);
    PRNU_CUDA_TRY(cudaLaunchKernel(fr.inv, g, b, args, fr.smem, s));
  }
  lc.n += 3;
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
