// internal.h -- host-side declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <tuple>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/prnu.h"
#include "common.cuh"

namespace prnu {

// ---------------------------------------------------------------- errors

struct Error {
  int code;
  std::string msg;
};
void set_error(const std::string& msg);
#define PRNU_CUDA_TRY(expr)                                                               \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess) throw ::prnu::Error{PRNU_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)}; \
  } while (0)
#define PRNU_CHECK_ARG(cond, what)                                                        \
  do {                                                                                    \
    if (!(cond)) throw ::prnu::Error{PRNU_EINVAL, what};                                  \
  } while (0)

// ---------------------------------------------------------------- plans

FftPlan make_plan(int n, const std::vector<int>& tw_offsets);
bool is_5smooth(int n);
// threads per row FFT and registers-per-thread class (1, 2 or 4 butterflies)
void row_launch_shape(const FftPlan& p, int* threads, int* maxb);
// threads per column block and butterflies per thread for 1 << lg columns
void col_launch_shape(const FftPlan& p, int lg, int* threads, int* maxb);

// ---------------------------------------------------------------- launchers (search.cu)

// Kernel kinds for per-kernel timing.
enum KernelKind {
  kKindResidual = 0, kKindFpSpectrum, kKindRowForward, kKindColumn, kKindRowInverse, kKindFinalize,
  kKindArgmax, kKindScatter, kKindNaiveWarp, kKindNaivePce, kKindFused, kKindCount
};
extern const char* const kKindNames[kKindCount];

// Counts every kernel launch; while profiling, brackets each launch with a
// pair of CUDA events recorded on the launching stream.
struct LaunchCounter {
  std::atomic<uint64_t> n{0};
  bool profiling = false;
  struct Rec {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  std::mutex mu;
  cudaEvent_t take();
  void start(int kind, cudaStream_t s);
  void stop(cudaStream_t s);
};

// RAII bracket around one launch (or a short fixed sequence of launches).
struct ProfScope {
  LaunchCounter& lc;
  cudaStream_t s;
  bool on;
  ProfScope(LaunchCounter& l, int kind, cudaStream_t st) : lc(l), s(st), on(l.profiling) {
    if (on) lc.start(kind, s);
  }
  ~ProfScope() {
    if (on) lc.stop(s);
  }
};

void launch_row_forward(const PassArgs& a, bool warp, const float* mean_sub, float2* out, cudaStream_t s,
                        LaunchCounter& lc);
// mode 0: forward FFT, multiply by the fingerprint, inverse FFT (in place)
// mode 1: forward FFT only, written to out_f32 / out_f16 scaled by *scale
// mode 2: multiply only by the fingerprint (packed spectra, in place)  [naive path]
// mode 3: forward only, in place (float2)                               [naive path]
// mode 4: inverse only, in place (float2)                               [naive path]
void launch_col(const PassArgs& a, int mode, float2* out_f32, void* out_f16, const float* scale,
                cudaStream_t s, LaunchCounter& lc);
void launch_row_inverse(const PassArgs& a, float* c_out, cudaStream_t s, LaunchCounter& lc);
void launch_finalize(const PassArgs& a, cudaStream_t s, LaunchCounter& lc);
// groups as SearchCall describes them (share = 1: contiguous)
void launch_argmax(const CandResult* res, const WorkItem* items, const int* group_start, int ngroups, int share,
                   prnu_result* out, const float* scale, int H, int W, cudaStream_t s, LaunchCounter& lc);
void launch_scatter_all(const CandResult* res, int nitems, int cmax, double* all, cudaStream_t s,
                        LaunchCounter& lc);
// fingerprint statistics: mean of K and the FP16 storage scale
void launch_fp_stats(const float* K, int H, int W, double* partials, int nblk, float* mean_out,
                     float* scale_out, float* inv_scale_out, bool half, cudaStream_t s, LaunchCounter& lc);
// naive path
void launch_naive_warp(const PassArgs& a, float* X, cudaStream_t s, LaunchCounter& lc);
void launch_naive_pce(const float* C, int H, int W, const WorkItem* item, const FpDesc* fps, const float* scale,
                      CandResult* out, float* blk_max, int* blk_arg, double* blk_sum, int nblk,
                      cudaStream_t s, LaunchCounter& lc);
void set_kernel_attributes();

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum
// minus the kernel's static shared memory (asking for more is rejected and
// leaves the 48 KB default in place).
template <class K>
inline void allow_max_dynamic_smem(K k) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, (const void*)k) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  cudaGetLastError();
}

// ---------------------------------------------------------------- launchers (residual.cu)

// Where residual pixel (y, x) of frame f is stored: f*fpitch + roff + y*rpitch + x.
struct ResidLayout {
  int rpitch;
  size_t fpitch;
  size_t roff;
};
// lay == nullptr: dense [F][H][W]
void launch_residual(const uint8_t* frames, int F, int H, int W, size_t pitch, int flags, int dtype, void* out,
                     float* scale, unsigned long long* acc, double* partials, int max_partials, cudaStream_t s,
                     LaunchCounter& lc, const ResidLayout* lay = nullptr);
size_t residual_partials_needed(int F, int H, int W);
// frame-literal residuals (Sec. 3.2): for render r of renders[nr] (frame
// index, similarity a11..a22) the residual of the warped uint8 frame, FP32,
// into out[r * lay.fpitch + lay.roff + y * lay.rpitch + x]; partials: at least
// literal_partials_needed(nr, H, W) doubles; nu2: nr floats; X: nr*H*W floats
// (the warped frames, scratch)
void launch_literal_residuals(const uint8_t* frames, size_t pitch, int H, int W, const WorkItem* renders, int nr,
                              int weight, float* out, const ResidLayout& lay, float* X, double* partials, float* nu2,
                              cudaStream_t s, LaunchCounter& lc);
size_t literal_partials_needed(int nr, int H, int W);
// s[f] = 1 / RMS from per-block sums of R^2 (nblk per frame); fill p[0..n) with v
void launch_resid_scale(const double* partials, int nblk, int F, int H, int W, float* scale, cudaStream_t s,
                        LaunchCounter& lc);
void launch_fill(float* p, int n, float v, cudaStream_t s, LaunchCounter& lc);
// residual by Mihcak's wavelet denoiser, `chunk` frames at a time through the
// scratch buffers bufA, bufT (chunk * Hp * Wp floats each, Hp, Wp = H, W
// rounded up to multiples of 16); partials: wavelet_partials_needed(F, H, W)
// doubles (PRNU_NORMALISE only); H, W >= 16
void launch_wavelet_residual(const uint8_t* frames, int F, int H, int W, size_t pitch, int flags, int dtype,
                             float sigma0, void* out, float* scale, float* bufA, float* bufT, int chunk,
                             double* partials, cudaStream_t s, LaunchCounter& lc);
size_t wavelet_partials_needed(int F, int H, int W);
// fingerprint resampling with T taps per axis: weights and (clamped) indices per output row and column
void launch_fp_resize(const float* K, size_t pitch, const float* wy, const int* iy, const float* wx, const int* ix,
                      int T, int H, int W, float* out, cudaStream_t s, LaunchCounter& lc);
// Eq. 2 accumulation over Lc residuals R [Lc][H][W] (R = I W(I)) and their frames
void launch_fp_estimate_accumulate(const float* R, const uint8_t* frames, size_t pitch, int Lc, int H, int W,
                                   double* num, double* den, bool first, cudaStream_t s, LaunchCounter& lc);
void launch_fp_estimate_divide(const double* num, const double* den, float* K, size_t n, cudaStream_t s,
                               LaunchCounter& lc);
// dense [F][H][W] residuals -> the zero-bordered layout the compile-time-planned
// kernels read (row pitch W + 3, pixel (0, 0) at W + 4, (H + 3)(W + 3) per frame)
// layout (half storage only): 0 single elements, 1 pairs (kF16P/kBF16P)
void launch_pad_frames(const void* in, int dtype, int F, int H, int W, void* out, cudaStream_t s, LaunchCounter& lc,
                       int layout = 0);
inline ResidLayout dense_layout(int H, int W) { return ResidLayout{W, (size_t)H * W, 0}; }
inline ResidLayout padded_layout(int H, int W) {
  return ResidLayout{W + 3, (size_t)(H + 3) * (W + 3), (size_t)(W + 3) + 1};
}

// ---------------------------------------------------------------- context

struct Fingerprint {
  int H = 0, W = 0;
  int dtype = kF32;
  void* d_spec = nullptr;    // spectrum, then (at tmap_off) the TMA descriptors of the column pass, if any
  size_t tmap_off = 0;       // 0: no descriptors
  float* d_scal = nullptr;   // [mean, scale, inv_scale]
  size_t bytes = 0;
  int refs = 0;
  cudaEvent_t ready = nullptr;
};

// the kernels' view of a cached fingerprint
inline FpDesc fp_desc(const Fingerprint& f) {
  return FpDesc{f.d_spec, f.dtype, f.d_scal + 2,
                f.tmap_off ? static_cast<const char*>(f.d_spec) + f.tmap_off : nullptr};
}

struct DeviceBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

class Server;

struct Tuning {
  int col_log2 = 3;   // generic kernels: columns per column-pass block = 1 << col_log2
  int ppb = 2;        // generic kernels: row pairs per row block
  int wave = 64;      // candidates in flight
  int variant = 0;    // compile-time-planned column variant; -1 = generic kernels only
  int persistent = 0; // compile-time-planned shapes: one persistent launch per call instead of waves
  int streams = 1;    // compile-time-planned shapes: waves alternate over 1 or 2 streams
  int share = 1;      // compile-time-planned shapes, waves: fingerprints of one (frame, node) share the forward pass
};

}  // namespace prnu

namespace prnu {
class BatchLoop;
}  // namespace prnu

struct prnu_ctx {
  int device = 0;
  int sm_count = 0;
  size_t budget = 0;
  std::atomic<size_t> used{0};
  std::recursive_mutex mu;
  std::map<uint64_t, std::shared_ptr<prnu::Fingerprint>> fps;
  uint64_t next_handle = 1;
  float2* d_tw = nullptr;
  std::vector<int> tw_off;   // offset per length, -1 if not 5-smooth
  prnu::LaunchCounter launches;
  cudaEvent_t last_done = nullptr;
  // call workspace
  prnu::DeviceBuf ws_spec, ws_stats, ws_items, ws_results, ws_groups, ws_out, ws_fpdesc, ws_misc, ws_resid,
      ws_persist, ws_pad, ws_fpest, ws_lit, ws_litx, ws_litpart, ws_renders, ws_resize, ws_wav, ws_corr;
  size_t tw_bytes = 0;
  int* h_err = nullptr;           // pinned: error flag of the last persistent launch or TMA wait
  int* d_err = nullptr;           // device flag the wave kernels raise when a bounded wait gives up
  int debug_stall = 0;            // prnu_debug_set(PRNU_DEBUG_STALL_DEVICE_WAITS)
  std::vector<char> h_stage;      // staging for host->device descriptors
  char* h_pinned = nullptr;
  size_t h_pinned_bytes = 0;
  cudaStream_t aux = nullptr;                    // the second stream of two-stream waves
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t stage_free = nullptr;
  std::map<std::pair<int, int>, prnu::Tuning> tuning;
  std::unique_ptr<prnu::Server> server;
  // eis_grid_search's device-resident loops (prnu_tuning.persistent = 2), by (H, W, residual layout)
  std::map<std::tuple<int, int, int>, std::unique_ptr<prnu::BatchLoop>> batch_loops;
  int server_loop = PRNU_LOOP_DEVICE;   // PRNU_LOOP_HOST / PRNU_LOOP_DEVICE, read when the server starts
};

namespace prnu {
// allocation helpers that honour the context budget
void* ctx_alloc(prnu_ctx* c, size_t bytes);
void ctx_free(prnu_ctx* c, void* p, size_t bytes);
void ensure_buf(prnu_ctx* c, DeviceBuf& b, size_t bytes);
// candidates per wave by default for frames of H x W: up to 1024, and up to 16 GB of spectra
int default_wave(int H, int W);
Tuning tuning_for(prnu_ctx* c, int H, int W);

// The search engine: enqueue the fused path for a prepared item list.
struct SearchCall {
  const void* resid;
  int rdtype;
  const float* scale;
  int F, H, W;
  std::vector<std::shared_ptr<Fingerprint>> fps;
  std::vector<WorkItem> items;
  // items of group g (= frame * P + fingerprint) are first + k * share for
  // k < count, with f = g / share, first = group_start[f] + g % share and
  // count = (group_start[f + 1] - group_start[f]) / share: share = 1, the
  // groups' items are contiguous ([F*P + 1] starts); share = P, the items
  // are ordered (frame, node, fingerprint) ([F + 1] starts) and every P
  // consecutive items form one forward unit
  std::vector<int> group_start;
  int share = 1;
  int cmax;
  bool prepadded = false;         // resid is FP32 in padded_layout already (zero border included)
};
// unit_major: order (frame, node, fingerprint) with call.share = P, else
// (frame, fingerprint, node) with call.share = 1
void build_items(const prnu_grid& g, const prnu_window* windows, int F, int P, SearchCall& call,
                 bool unit_major = false);
// whether eis_grid_search-style calls of P fingerprints on H x W share the forward pass
bool share_forward(prnu_ctx* c, int H, int W, int P, bool naive);
void validate_shape(int H, int W);
// enqueue: results into d_out (device prnu_result [F*P]); optional d_all
void enqueue_search(prnu_ctx* c, const SearchCall& call, prnu_result* d_out, double* d_all, bool naive,
                    cudaStream_t s);

}  // namespace prnu
