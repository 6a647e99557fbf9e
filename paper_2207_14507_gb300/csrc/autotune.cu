// autotune.cu -- prnu_autotune: pick the column-pass variant and the wave size
// of the fused path for one frame size by timing them on synthetic data.
#include <algorithm>
#include <chrono>

#include "internal.h"
#include "search_fixed.h"

namespace prnu {

namespace {

// counter-based uniform noise in [-1, 1): a 64-bit mix of (seed, index)
__global__ void k_fill_noise(float* __restrict__ p, size_t n, unsigned long long seed) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    p[i] = (float)((double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
  }
}

}  // namespace

}  // namespace prnu

using namespace prnu;

extern "C" int prnu_autotune(prnu_ctx* ctx, int H, int W, int dtype, double budget_ms, prnu_tuning* best,
                             prnu_stream stream) {
  if (!ctx) {
    set_error("NULL context");
    return PRNU_EINVAL;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device) cudaSetDevice(ctx->device);
  int code = PRNU_OK;
  void* resid = nullptr;
  size_t resid_bytes = 0;
  float* K = nullptr;
  uint64_t h = 0;
  try {
    validate_shape(H, W);
    PRNU_CHECK_ARG(dtype == kF32 || dtype == kF16 || dtype == kBF16, "unknown dtype");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int F = 2;
    const size_t px = (size_t)H * W;
    // synthetic residual (FP32 noise, stored in the requested type) and fingerprint
    resid_bytes = F * px * sizeof(float);
    resid = ctx_alloc(ctx, resid_bytes);
    K = reinterpret_cast<float*>(ctx_alloc(ctx, px * sizeof(float)));
    k_fill_noise<<<512, 256, 0, s>>>(reinterpret_cast<float*>(resid), F * px, 12345ull);
    k_fill_noise<<<512, 256, 0, s>>>(K, px, 999ull);
    PRNU_CUDA_TRY(cudaGetLastError());
    int rc = prnu_fingerprint_term(ctx, K, H, W, dtype == kF32 ? kF32 : kF16, &h, stream);
    if (rc != PRNU_OK) throw Error{rc, prnu_last_error()};
    Tuning base = tuning_for(ctx, H, W);
    const FixedShape* fs = find_fixed(H, W);
    const size_t per_item = (size_t)H * (W / 2) * sizeof(float2) + (size_t)H * sizeof(RowStat);
    // waves: a few small ones, then the size's default (up to 1024 candidates,
    // 16 GB of spectra).  The timed search below has 512 candidates, so larger
    // waves cannot be told apart there; the default is taken for them
    std::vector<int> waves;
    const int def_wave = default_wave(H, W);
    for (int w : {16, 64, 128, 256, def_wave})
      if (w <= def_wave && (size_t)w * per_item < ctx->budget / 4 &&
          std::find(waves.begin(), waves.end(), w) == waves.end())
        waves.push_back(w);
    if (waves.empty()) waves.push_back(1);
    // candidate configurations: generic kernels and every compile-time column
    // variant and row-pair count, each over the wave sizes, and the persistent launch
    std::vector<Tuning> configs;
    for (int w : waves) {
      Tuning t = base;
      t.variant = -1;
      t.persistent = 0;
      t.wave = w;
      configs.push_back(t);
    }
    if (fs) {
      for (const FixedRow& r : fs->rows) {
        if (!fixed_supports(*fs, H, r.ppb)) continue;
        for (int v = 0; v < (int)fs->cols.size(); ++v)
          for (int w : waves) {
            Tuning t = base;
            t.variant = v;
            t.ppb = r.ppb;
            t.persistent = 0;
            t.wave = w;
            configs.push_back(t);
          }
      }
      if ((size_t)kPersistSlots * per_item < ctx->budget / 4) {
        Tuning t = base;
        t.variant = 0;
        t.ppb = fs->rows.front().ppb;
        t.persistent = 1;
        configs.push_back(t);
      }
    }
    // 16 x 16 grid nodes per frame: 512 candidates per timed search
    prnu_grid g{0.95f, 0.00625f, 16, -2.0f, 0.25f, 16};
    const int rdt = kF32;   // the timed residual is FP32 noise whatever the storage type
    cudaEvent_t e0, e1;
    PRNU_CUDA_TRY(cudaEventCreate(&e0));
    PRNU_CUDA_TRY(cudaEventCreate(&e1));
    Tuning winner = base;
    double best_ms = 1e300;
    const auto t_start = std::chrono::steady_clock::now();
    std::vector<prnu_result> out(F);
    prnu_result* d_out = nullptr;
    ensure_buf(ctx, ctx->ws_out, sizeof(prnu_result) * F);
    d_out = reinterpret_cast<prnu_result*>(ctx->ws_out.p);
    SearchCall call;
    call.resid = resid;
    call.rdtype = rdt;
    call.scale = nullptr;
    call.F = F;
    call.H = H;
    call.W = W;
    call.fps.push_back(ctx->fps.at(h));
    build_items(g, nullptr, F, 1, call);
    for (const Tuning& t : configs) {
      const double spent =
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
      if (spent > budget_ms && best_ms < 1e300) break;
      ctx->tuning[{H, W}] = t;
      enqueue_search(ctx, call, d_out, nullptr, false, s);   // warm-up
      float ms = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {                    // best of two
        PRNU_CUDA_TRY(cudaEventRecord(e0, s));
        enqueue_search(ctx, call, d_out, nullptr, false, s);
        PRNU_CUDA_TRY(cudaEventRecord(e1, s));
        PRNU_CUDA_TRY(cudaEventSynchronize(e1));
        float m = 0.f;
        PRNU_CUDA_TRY(cudaEventElapsedTime(&m, e0, e1));
        ms = std::min(ms, m);
      }
      if (*ctx->h_err) {   // a bounded device-side wait gave up: never pick this configuration
        *ctx->h_err = 0;
        PRNU_CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s));
        continue;
      }
      if (ms < best_ms) {
        best_ms = ms;
        winner = t;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tuning[{H, W}] = winner;
    if (best) {
      best->col_width = 1 << winner.col_log2;
      best->pairs_per_block = winner.ppb;
      best->wave = winner.wave;
      best->variant = winner.variant;
      best->persistent = winner.persistent;
      best->streams = winner.streams;
      best->share_forward = winner.share;
    }
  } catch (const Error& e) {
    set_error(e.msg);
    code = e.code;
  }
  if (h) prnu_fingerprint_release(ctx, h);
  cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
  if (resid) ctx_free(ctx, resid, resid_bytes);
  if (K) ctx_free(ctx, K, (size_t)H * W * sizeof(float));
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  if (code == PRNU_OK) set_error("");
  return code;
}
