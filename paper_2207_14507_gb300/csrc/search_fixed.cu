// search_fixed.cu -- compile-time-planned kernels of the grid search for the
// frame sizes of the workloads (256x256, 1280x720, 1920x1080, 3840x2160).
//
// Same arithmetic as the generic kernels in search.cu (the same Stockham
// stages and radix-R DFTs, the same packed half spectrum), with the plan known
// at compile time and fewer shared-memory passes:
//   k_row_forward_fx : stage 0 of the row FFT takes its inputs straight from
//                      the bilinear warp (no shared-memory fill);
//   k_col_fx         : stage 0 loads the strip from global memory; the last
//                      forward stage, the spectrum product and the first
//                      inverse stage stay in registers (the inverse plan is
//                      the forward plan reversed, so every thread already
//                      holds its inputs); the last inverse stage stores to
//                      global memory; stages in between run in place;
//   k_row_inverse_fx : stage 0 rebuilds the two rows' full spectrum straight
//                      from global memory; the last stage's outputs are
//                      reduced to the row statistics from registers.
#include <float.h>
#include <limits.h>

#include "fft_fixed.cuh"
#include "internal.h"
#include "search_fixed.h"

namespace prnu {

namespace {

struct WarpRedF {
  float ma;
  int ia;
  float mb;
  int ib;
  double sa;
  double sb;
};

__device__ __forceinline__ void better_fx(float& v, int& i, float v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) {
    v = v2;
    i = i2;
  }
}

template <int DT>
__device__ __forceinline__ float bilinear_fx(const void* R, size_t base, int H, int W, float qx, float qy) {
  const float fx0 = floorf(qx), fy0 = floorf(qy);
  const float fx = qx - fx0, fy = qy - fy0;
  const int x0 = (int)fx0, y0 = (int)fy0;
  const bool xi0 = (unsigned)x0 < (unsigned)W, xi1 = (unsigned)(x0 + 1) < (unsigned)W;
  const bool yi0 = (unsigned)y0 < (unsigned)H, yi1 = (unsigned)(y0 + 1) < (unsigned)H;
  const size_t r0 = base + (size_t)y0 * W + x0;
  const float v00 = (yi0 && xi0) ? load_store_type<DT>(R, r0) : 0.f;
  const float v01 = (yi0 && xi1) ? load_store_type<DT>(R, r0 + 1) : 0.f;
  const float v10 = (yi1 && xi0) ? load_store_type<DT>(R, r0 + W) : 0.f;
  const float v11 = (yi1 && xi1) ? load_store_type<DT>(R, r0 + W + 1) : 0.f;
  const float gx = 1.f - fx, gy = 1.f - fy;
  return gy * (gx * v00 + fx * v01) + fy * (gx * v10 + fx * v11);
}

// full spectrum element i of z = G_a + i G_b from two packed rows
struct FullRowLd {
  const float2* pa;
  const float2* pb;
  int W, Wh;
  __device__ __forceinline__ float2 operator()(int i, int) const {
    if (i == 0) {
      const float2 A = pa[0], B = pb[0];
      return make_float2(A.x, B.x);
    }
    if (i == Wh) {
      const float2 A = pa[0], B = pb[0];
      return make_float2(A.y, B.y);
    }
    if (i < Wh) {
      const float2 A = pa[i], B = pb[i];
      return make_float2(A.x - B.y, A.y + B.x);
    }
    const int k = W - i;
    const float2 A = pa[k], B = pb[k];
    return make_float2(A.x + B.y, B.x - A.y);
  }
};

struct StripLd {
  const float2* Z;
  int Wh, c0;
  __device__ __forceinline__ float2 operator()(int i, int c) const {
    const int col = c0 + c;
    return col < Wh ? Z[(size_t)i * Wh + col] : make_float2(0.f, 0.f);
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
  return (size_t)ppb * 2 * row_smem_len(W) * sizeof(float2) + (size_t)ppb * 32 * sizeof(WarpRedF);
}

// ---------------------------------------------------------------- row forward

template <int DT, class SP, int T, int PPB>
__global__ void __launch_bounds__(T * PPB) k_row_forward_fx(PassArgs a) {
  constexpr int W = SP::N, Wh = W / 2, L = row_smem_len(W);
  extern __shared__ float2 smem[];
  const int grp = threadIdx.x / T, t = threadIdx.x - grp * T;
  const int H = a.H;
  const int pair = blockIdx.x * PPB + grp;
  const int slot = blockIdx.y;
  float2* A = smem + (size_t)grp * 2 * L;
  float2* B = A + L;
  const float2* tw = a.tw + a.prow.tw_off;
  const WorkItem it = item_of(a, slot);
  size_t base;
  const void* Rf = frame_of(a, it.frame, &base);
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
      v[r].x = bilinear_fx<DT>(Rf, base, H, W, fmaf(it.a11, dx, bx0), fmaf(it.a21, dx, by0));
      v[r].y = bilinear_fx<DT>(Rf, base, H, W, fmaf(it.a11, dx, bx1), fmaf(it.a21, dx, by1));
    }
    Dft<S0::R, false>::run(v);
#pragma unroll
    for (int r = 0; r < S0::R; ++r) A[rpad(j * S0::R + r)] = v[r];
  }
  __syncthreads();
  const float2* res = RowStagesPP<SP, 1, SP::S, T, false>::run(A, B, t, tw);
  float2* o0 = a.spec + ((size_t)slot * H + y0) * Wh;
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

template <class SP, int NC, int T>
__global__ void __launch_bounds__(T) k_col_fx(PassArgs a) {
  constexpr int H = SP::N;
  using IS = typename SP::Rev;
  extern __shared__ float2 sm[];
  const int t = threadIdx.x;
  const int Wh = a.W >> 1;
  const int c0 = blockIdx.x * NC;
  const int slot = blockIdx.y;
  float2* Z = a.spec + (size_t)slot * H * Wh;
  const float2* tw = a.tw + a.pcol.tw_off;
  const WorkItem wi = item_of(a, slot);
  const FpDesc fp = a.fps[wi.fp];

  stage_stream<StageC<SP, 0, T, NC>, false>(t, tw, StripLd{Z, Wh, c0}, ColSt<NC>{sm});
  __syncthreads();
  ColStagesIP<SP, 1, SP::S - 1, T, NC, false>::run(sm, t, tw);

  using FL = StageC<SP, SP::S - 1, T, NC>;
  using I0 = StageC<IS, 0, T, NC>;
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
      const float2 S = load_spec(fp.spec, fp.dtype, (size_t)(j + r * FL::NS) * Wh + col);
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

template <class SP, int T, int PPB>
__global__ void __launch_bounds__(T * PPB) k_row_inverse_fx(PassArgs a) {
  constexpr int W = SP::N, Wh = W / 2, L = row_smem_len(W);
  extern __shared__ float2 smem[];
  const int grp = threadIdx.x / T, t = threadIdx.x - grp * T;
  const int H = a.H;
  const int pair = blockIdx.x * PPB + grp;
  const int slot = blockIdx.y;
  float2* A = smem + (size_t)grp * 2 * L;
  float2* B = A + L;
  WarpRedF* red = reinterpret_cast<WarpRedF*>(smem + (size_t)PPB * 2 * L) + grp * 32;
  const float2* tw = a.tw + a.prow.tw_off;
  const float2* pa = a.spec + ((size_t)slot * H + 2 * pair) * Wh;
  stage_stream<StageC<SP, 0, T>, true>(t, tw, FullRowLd{pa, pa + Wh, W, Wh}, RowSt{A});
  __syncthreads();
  const float2* res = RowStagesPP<SP, 1, SP::S - 1, T, true>::run(A, B, t, tw);
  using SL = StageC<SP, SP::S - 1, T>;
  static_assert(SL::NB == SL::NS, "last stage writes j + r*NS");
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
      better_fx(ma, ia, v.x, x);
      better_fx(mb, ib, v.y, x);
      sa = fmaf(v.x, v.x, sa);
      sb = fmaf(v.y, v.y, sb);
    }
  }
  double da = sa, db = sb;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    float m2 = __shfl_xor_sync(0xffffffffu, ma, o);
    int i2 = __shfl_xor_sync(0xffffffffu, ia, o);
    better_fx(ma, ia, m2, i2);
    m2 = __shfl_xor_sync(0xffffffffu, mb, o);
    i2 = __shfl_xor_sync(0xffffffffu, ib, o);
    better_fx(mb, ib, m2, i2);
    da += __shfl_xor_sync(0xffffffffu, da, o);
    db += __shfl_xor_sync(0xffffffffu, db, o);
  }
  const int w = t >> 5;
  if ((t & 31) == 0) red[w] = WarpRedF{ma, ia, mb, ib, da, db};
  __syncthreads();
  if (t == 0) {
    constexpr int NW = (T + 31) / 32;
    for (int k = 1; k < NW; ++k) {
      better_fx(ma, ia, red[k].ma, red[k].ia);
      better_fx(mb, ib, red[k].mb, red[k].ib);
      da += red[k].sa;
      db += red[k].sb;
    }
    RowStat* st = a.stats + (size_t)slot * H + 2 * pair;
    st[0] = RowStat{ma, ia, da};
    st[1] = RowStat{mb, ib, db};
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
  static FixedShape make(std::vector<FixedRow> rows, std::vector<FixedCol> cols) {
    FixedShape s{};
    s.W = W;
    s.H = H;
    s.rows = std::move(rows);
    s.cols = std::move(cols);
    return s;
  }
};

std::vector<FixedShape> build_registry() {
  std::vector<FixedShape> v;
  {
    using D = ShapeDef<Spec<1920, 16, 12, 10>, 192, Spec<1080, 12, 10, 9>>;
    v.push_back(D::make({D::row<2>(), D::row<1>()},
                        {D::col<4, 480>(), D::col<8, 480>(), D::col<8, 960>(), D::col<16, 960>()}));
  }
  {
    using D = ShapeDef<Spec<1280, 16, 10, 8>, 160, Spec<720, 10, 9, 8>>;
    v.push_back(D::make({D::row<2>(), D::row<1>()}, {D::col<4, 384>(), D::col<8, 384>(), D::col<16, 736>()}));
  }
  {
    using D = ShapeDef<Spec<3840, 16, 16, 15>, 256, Spec<2160, 15, 12, 12>>;
    v.push_back(D::make({D::row<2>(), D::row<1>()}, {D::col<4, 384>(), D::col<4, 736>(), D::col<8, 736>()}));
  }
  {
    using D = ShapeDef<Spec<256, 16, 16>, 32, Spec<256, 16, 16>>;
    v.push_back(D::make({D::row<4>(), D::row<2>()}, {D::col<8, 128>(), D::col<16, 256>()}));
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

}  // namespace prnu
