// api.cu -- C ABI of libprnu (see include/prnu.h): context, FFT plans and
// twiddle table, fingerprint-spectrum cache, work lists and the search driver.
#include <climits>
#include <cmath>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <functional>

#include "internal.h"
#include "wave_loop.h"
#include "search_fixed.h"
#include "server.h"

namespace prnu {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

template <class Fn>
int guarded(Fn&& fn) {
  try {
    fn();
    g_last_error.clear();
    return PRNU_OK;
  } catch (const Error& e) {
    g_last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return PRNU_ENOMEM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return PRNU_EINVAL;
  }
}

const int kRadices[] = {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};

void plan_search(int n, int maxr, std::vector<int>& cur, std::vector<int>& best) {
  if (n == 1) {
    if (best.empty() || cur.size() < best.size() || (cur.size() == best.size() && cur.back() > best.back()))
      best = cur;
    return;
  }
  if (!best.empty() && cur.size() + 1 > best.size()) return;
  for (int r : kRadices) {
    if (r > maxr || n % r) continue;
    cur.push_back(r);
    plan_search(n / r, r, cur, best);
    cur.pop_back();
  }
}

int roundup32(int v) { return (v + 31) & ~31; }

}  // namespace

bool is_5smooth(int n) {
  if (n < 1) return false;
  for (int p : {2, 3, 5})
    while (n % p == 0) n /= p;
  return n == 1;
}

FftPlan make_plan(int n, const std::vector<int>& tw_offsets) {
  FftPlan p{};
  PRNU_CHECK_ARG(n >= 2 && n <= kMaxFft && is_5smooth(n), "FFT length must be 5-smooth in [2, 4096]");
  std::vector<int> cur, best;
  plan_search(n, 16, cur, best);
  PRNU_CHECK_ARG(!best.empty() && (int)best.size() <= kMaxStages, "no FFT plan");
  p.n = n;
  p.nstages = (int)best.size();
  for (int i = 0; i < p.nstages; ++i) p.radix[i] = best[i];
  p.min_radix = best.back();
  p.tw_off = tw_offsets[n];
  return p;
}

void row_launch_shape(const FftPlan& p, int* threads, int* maxb) {
  // one thread per butterfly of the stage with the most butterflies, at most 256
  const int nb = p.n / p.min_radix;
  *threads = std::min(256, std::max(32, roundup32(nb)));
  *maxb = 1;
}

void col_launch_shape(const FftPlan& p, int lg, int* threads, int* maxb) {
  const int total = (p.n / p.min_radix) << lg;
  *threads = std::min(512, std::max(32, roundup32(total)));
  *maxb = 1;
}

void validate_shape(int H, int W) {
  PRNU_CHECK_ARG(H >= 16 && W >= 16 && H <= kMaxFft && W <= kMaxFft, "H and W must lie in [16, 4096]");
  PRNU_CHECK_ARG(H % 2 == 0 && W % 2 == 0, "H and W must be even");
  PRNU_CHECK_ARG(is_5smooth(H) && is_5smooth(W), "H and W must be 5-smooth (factors 2, 3, 5 only)");
}

void* ctx_alloc(prnu_ctx* c, size_t bytes) {
  if (bytes == 0) return nullptr;
  if (c->used.load() + bytes > c->budget)
    throw Error{PRNU_ENOMEM, "HBM budget exceeded (" + std::to_string(c->used.load() + bytes) + " > " +
                                 std::to_string(c->budget) + " bytes)"};
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    throw Error{PRNU_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed"};
  }
  c->used += bytes;
  return p;
}

void ctx_free(prnu_ctx* c, void* p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  c->used -= bytes;
}

void ensure_buf(prnu_ctx* c, DeviceBuf& b, size_t bytes) {
  if (b.bytes >= bytes) return;
  // the old buffer may still be in use by enqueued work
  if (b.p) {
    PRNU_CUDA_TRY(cudaEventSynchronize(c->last_done));
    ctx_free(c, b.p, b.bytes);
    b.p = nullptr;
    b.bytes = 0;
  }
  size_t want = std::max(bytes, (size_t)4096);
  b.p = ctx_alloc(c, want);
  b.bytes = want;
}

int default_wave(int H, int W) {
  const size_t per_item = (size_t)H * (W / 2) * sizeof(float2) + (size_t)H * sizeof(RowStat);
  return (int)std::max<size_t>(1, std::min<size_t>(1024, ((size_t)16 << 30) / per_item));
}

Tuning tuning_for(prnu_ctx* c, int H, int W) {
  auto it = c->tuning.find({H, W});
  if (it != c->tuning.end()) return it->second;
  Tuning t;
  FftPlan pc = make_plan(H, c->tw_off);
  t.col_log2 = 0;
  for (int lg = 4; lg >= 0; --lg) {
    const size_t sm = 2 * (size_t)H * (1u << lg) * sizeof(float2);
    if (sm <= 112 * 1024) {
      t.col_log2 = lg;
      break;
    }
  }
  // the planned kernels run one row pair per block best; waves of up to 1024
  // candidates (up to 16 GB of spectra) amortise the per-wave finalisation and
  // tail: 1024 against 512 gains 0.7% at 1080p, 512 against 129 1% at 4K
  t.ppb = find_fixed(H, W) ? 1 : 2;
  // sizes without compile-time-planned kernels run the generic ones (-1), so
  // that what prnu_get_tuning reports is accepted by prnu_set_tuning
  t.variant = find_fixed(H, W) ? 0 : -1;
  // within a quarter of the context's HBM budget (spectra and row statistics)
  const size_t per_item = (size_t)H * (W / 2) * sizeof(float2) + (size_t)H * sizeof(RowStat);
  t.wave = (int)std::max<size_t>(1, std::min<size_t>((size_t)default_wave(H, W), c->budget / 4 / per_item));
  // one stream: two-stream waves gain under 1% at 1080p and make the
  // per-launch event times overlap (prnu_set_tuning selects them)
  t.streams = 1;
  return t;
}

bool share_forward(prnu_ctx* c, int H, int W, int P, bool naive) {
  if (naive || P < 2) return false;
  const Tuning t = tuning_for(c, H, W);
  if (!t.share || t.persistent == 1 || t.variant < 0 || P > t.wave) return false;
  const FixedShape* fs = find_fixed(H, W);
  return fs && fixed_supports(*fs, H, t.ppb);
}

// Host-side staging of small descriptor arrays through pinned memory.
struct Stager {
  prnu_ctx* c;
  size_t off = 0;
  std::vector<std::function<void(char*)>> writers;
  struct Copy {
    void* dst;
    size_t off, bytes;
  };
  std::vector<Copy> copies;
  explicit Stager(prnu_ctx* ctx) : c(ctx) {}
  template <class T>
  void add(void* dst, const T* src, size_t count) {
    const size_t bytes = sizeof(T) * count;
    if (!bytes) return;
    const size_t o = off;
    copies.push_back(Copy{dst, o, bytes});
    writers.push_back([=](char* base) { memcpy(base + o, src, bytes); });
    off = (off + bytes + 255) & ~(size_t)255;
  }
  void flush(cudaStream_t s) {
    if (copies.empty()) return;
    PRNU_CUDA_TRY(cudaEventSynchronize(c->stage_free));
    if (c->h_pinned_bytes < off) {
      if (c->h_pinned) cudaFreeHost(c->h_pinned);
      c->h_pinned = nullptr;
      c->h_pinned_bytes = 0;
      size_t want = std::max(off, (size_t)1 << 20);
      PRNU_CUDA_TRY(cudaHostAlloc((void**)&c->h_pinned, want, cudaHostAllocDefault));
      c->h_pinned_bytes = want;
    }
    for (auto& w : writers) w(c->h_pinned);
    for (auto& cp : copies)
      PRNU_CUDA_TRY(cudaMemcpyAsync(cp.dst, c->h_pinned + cp.off, cp.bytes, cudaMemcpyHostToDevice, s));
    PRNU_CUDA_TRY(cudaEventRecord(c->stage_free, s));
  }
};

void build_items(const prnu_grid& g, const prnu_window* windows, int F, int P, SearchCall& call, bool unit_major) {
  PRNU_CHECK_ARG(g.nlam >= 1 && g.nth >= 1, "grid must have nlam >= 1 and nth >= 1");
  PRNU_CHECK_ARG((long long)g.nlam * g.nth <= (1 << 24), "grid too large");
  call.items.clear();
  call.share = unit_major ? P : 1;
  call.group_start.assign((size_t)F * (unit_major ? 1 : P) + 1, 0);
  call.cmax = g.nlam * g.nth;
  std::vector<float> lam(g.nlam), th(g.nth);
  for (int i = 0; i < g.nlam; ++i) lam[i] = (float)((double)g.lam0 + (double)i * (double)g.dlam);
  for (int j = 0; j < g.nth; ++j) th[j] = (float)((double)g.th0_deg + (double)j * (double)g.dth_deg);
  for (int f = 0; f < F; ++f) {
    int il = 0, ih = g.nlam - 1, jl = 0, jh = g.nth - 1;
    if (windows) {
      const prnu_window& w = windows[f];
      PRNU_CHECK_ARG(w.lam_lo >= 0 && w.lam_lo <= w.lam_hi && w.lam_hi < g.nlam && w.th_lo >= 0 &&
                         w.th_lo <= w.th_hi && w.th_hi < g.nth,
                     "window " + std::to_string(f) + " lies outside the grid");
      il = w.lam_lo; ih = w.lam_hi; jl = w.th_lo; jh = w.th_hi;
    }
    auto node = [&](int p, int i, int j) {
      const double L = (double)lam[i];
      PRNU_CHECK_ARG(L > 0 && std::isfinite(L), "grid scales must be positive");
      const double t = (double)th[j] * 3.14159265358979323846 / 180.0;
      const double cs = cos(t), sn = sin(t);
      WorkItem it;
      it.frame = f;
      it.fp = p;
      it.cand = i * g.nth + j;
      it.group = f * P + p;
      it.a11 = (float)(cs / L);
      it.a12 = (float)(sn / L);
      it.a21 = (float)(-sn / L);
      it.a22 = (float)(cs / L);
      it.lam = lam[i];
      it.th_deg = th[j];
      call.items.push_back(it);
    };
    if (unit_major) {
      call.group_start[f] = (int)call.items.size();
      for (int i = il; i <= ih; ++i)
        for (int j = jl; j <= jh; ++j)
          for (int p = 0; p < P; ++p) node(p, i, j);
    } else {
      for (int p = 0; p < P; ++p) {
        call.group_start[(size_t)f * P + p] = (int)call.items.size();
        for (int i = il; i <= ih; ++i)
          for (int j = jl; j <= jh; ++j) node(p, i, j);
      }
    }
  }
  call.group_start.back() = (int)call.items.size();
  PRNU_CHECK_ARG(call.items.size() < (size_t)INT_MAX, "too many candidates");
}

static std::vector<FpDesc> fp_descs(const SearchCall& call) {
  std::vector<FpDesc> d;
  for (auto& f : call.fps) d.push_back(fp_desc(*f));
  return d;
}

// A bounded device-side wait (a TMA copy of the column pass, a dependency of
// the persistent kernel) gave up: clear both flags and fail the call.
[[noreturn]] static void report_device_abort(prnu_ctx* c, cudaStream_t s, const char* what) {
  *c->h_err = 0;
  PRNU_CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), s));
  throw Error{PRNU_EDEVICE_ABORT, what};
}

void enqueue_search(prnu_ctx* c, const SearchCall& call, prnu_result* d_out, double* d_all, bool naive,
                    cudaStream_t s) {
  const int H = call.H, W = call.W, Wh = W / 2;
  const int n = (int)call.items.size();
  const int share = std::max(call.share, 1);
  const int ngroups = ((int)call.group_start.size() - 1) * share;
  const FftPlan prow = make_plan(W, c->tw_off), pcol = make_plan(H, c->tw_off);
  Tuning tn = tuning_for(c, H, W);
  int rowT, rowMB;
  row_launch_shape(prow, &rowT, &rowMB);
  // waves hold whole forward units (share items each)
  const int wave = naive ? 1 : std::max(share, std::min(tn.wave, n) / share * share);
  const FixedShape* fs = (!naive && tn.variant >= 0) ? find_fixed(H, W) : nullptr;
  if (fs && !fixed_supports(*fs, H, tn.ppb)) fs = nullptr;
  PRNU_CHECK_ARG(share == 1 || (fs && tn.persistent != 1 && n % share == 0),
                 "shared forward units need the compile-time-planned wave kernels");
  bool persistent = fs && tn.persistent == 1 && (H / 2) % fs->persist.ppb == 0;
  // the device-resident loop: every wave of the call in one graph launch
  const bool graph = fs && tn.persistent == 2 && !naive && !call.prepadded;
  if (persistent) {   // tickets of one launch: (n + 3) steps of 2 row phases, the column phase and a finalisation
    const long long nrf = (H / 2) / fs->persist.ppb, ncol = (Wh + fs->persist.nc - 1) / fs->persist.nc;
    persistent = (long long)(n + 3) * (2 * nrf + ncol + 1) < (long long)INT_MAX;
  }
  // two-stream waves: alternate waves on s and the context's second stream,
  // each on its own half of the workspace
  const bool two = fs && !persistent && !graph && !naive && tn.streams == 2 && n > wave && share == 1;
  // forward units compute in slots after the wave's candidates (one per unit)
  const int slots = persistent ? kPersistSlots : (two ? 2 * wave : wave + (share > 1 ? wave / share : 0));

  if (*c->h_err)   // a bounded wait of an earlier asynchronous call gave up
    report_device_abort(c, s, "a bounded device-side wait of an earlier call timed out; its results are invalid");
  PRNU_CUDA_TRY(cudaStreamWaitEvent(s, c->last_done, 0));
  for (auto& f : call.fps) PRNU_CUDA_TRY(cudaStreamWaitEvent(s, f->ready, 0));
  ensure_buf(c, c->ws_items, sizeof(WorkItem) * std::max(n, 1));
  ensure_buf(c, c->ws_results, sizeof(CandResult) * std::max(n, 1));
  ensure_buf(c, c->ws_groups, sizeof(int) * (ngroups + 1));
  ensure_buf(c, c->ws_fpdesc, sizeof(FpDesc) * std::max<size_t>(1, call.fps.size()));
  ensure_buf(c, c->ws_spec, (size_t)slots * H * Wh * sizeof(float2));
  ensure_buf(c, c->ws_stats, (size_t)slots * H * sizeof(RowStat));
  if (persistent) ensure_buf(c, c->ws_persist, sizeof(int) * (2 + 4 * (size_t)n));
  // the compile-time-planned kernels read the residuals in the zero-bordered
  // layout; residuals rendered in it already (prepadded) serve both paths
  PRNU_CHECK_ARG(!call.prepadded || (call.rdtype == kF32 && !naive), "prepadded residuals are FP32, planned or generic");
  const ResidLayout lay = (fs || call.prepadded) ? padded_layout(H, W) : dense_layout(H, W);
  const bool pad = fs && !call.prepadded;
  // half storage for the wave kernels: the pair layout (one load per row and sample)
  // half storage for the wave kernels: the pair layout (one load per row and sample)
  const bool pairs = pad && !persistent && call.rdtype != kF32;
  if (pad) ensure_buf(c, c->ws_pad, (size_t)call.F * lay.fpitch * (call.rdtype == kF32 || pairs ? 4 : 2));
  std::vector<FpDesc> fd = fp_descs(call);
  Stager st(c);
  st.add(c->ws_items.p, call.items.data(), call.items.size());
  st.add(c->ws_groups.p, call.group_start.data(), call.group_start.size());
  st.add(c->ws_fpdesc.p, fd.data(), fd.size());
  st.flush(s);

  PassArgs a{};
  a.resid = call.resid;
  if (pad) {
    launch_pad_frames(call.resid, call.rdtype, call.F, H, W, c->ws_pad.p, s, c->launches, pairs ? 1 : 0);
    a.resid = c->ws_pad.p;
  }
  a.rdtype = pairs ? (call.rdtype == kF16 ? kF16P : kBF16P) : call.rdtype;
  a.rpitch = lay.rpitch;
  a.fpitch = lay.fpitch;
  a.roff = lay.roff;
  a.H = H;
  a.W = W;
  a.items = reinterpret_cast<const WorkItem*>(c->ws_items.p);
  a.spec = reinterpret_cast<float2*>(c->ws_spec.p);
  a.stats = reinterpret_cast<RowStat*>(c->ws_stats.p);
  a.results = reinterpret_cast<CandResult*>(c->ws_results.p);
  a.fps = reinterpret_cast<const FpDesc*>(c->ws_fpdesc.p);
  a.scale = call.scale;
  a.tw = c->d_tw;
  a.prow = prow;
  a.pcol = pcol;
  a.err = c->d_err;
  a.stall = c->debug_stall;
  a.pairs_per_block = naive ? 2 : tn.ppb;
  a.col_log2 = tn.col_log2;
  a.row_threads = rowT;
  a.share = share;
  a.units = nullptr;
  a.unit_of = nullptr;
  a.fp_f32 = std::any_of(fd.begin(), fd.end(), [](const FpDesc& d) { return d.dtype == kF32; }) ? 1 : 0;

  if (graph) {
    auto& bl = c->batch_loops[std::make_tuple(H, W, (int)a.rdtype)];
    if (!bl) bl.reset(new BatchLoop(c));
    WaveLoopConfig g;
    g.fs = fs;
    g.variant = tn.variant;
    g.ppb = tn.ppb;
    g.col_log2 = tn.col_log2;
    g.H = H;
    g.W = W;
    g.rdtype = a.rdtype;
    g.wave = std::min(wave, kLoopMaxWave / share * share);
    g.fp_f32 = a.fp_f32;
    g.spec = a.spec;
    g.stats = a.stats;
    g.spec_slots = slots;
    g.resid = a.resid;
    g.fps = a.fps;
    g.scale = a.scale;
    g.err = a.err;
    g.stall = a.stall;
    DevRun r{};
    r.items = a.items;
    r.results = a.results;
    r.groups = reinterpret_cast<const int*>(c->ws_groups.p);
    r.n = n;
    r.share = share;
    r.ngroups = 0;   // the arg-max runs after the loop, as for the other paths
    bl->run(g, r, s);
    PRNU_CUDA_TRY(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  } else if (persistent) {
    int* st0 = reinterpret_cast<int*>(c->ws_persist.p);
    PersistArgs p{st0, st0 + 1, st0 + 2, st0 + 2 + n, st0 + 2 + 2 * (size_t)n, st0 + 2 + 3 * (size_t)n, n,
                  kPersistSlots};
    PRNU_CUDA_TRY(cudaMemsetAsync(st0, 0, sizeof(int) * (2 + 4 * (size_t)n), s));
    a.item0 = 0;
    a.nitems = n;
    launch_persistent(a, p, *fs, c->sm_count, s, c->launches);
    PRNU_CUDA_TRY(cudaMemcpyAsync(c->h_err, p.error, sizeof(int), cudaMemcpyDeviceToHost, s));
  } else if (two) {
    if (!c->aux) {
      PRNU_CUDA_TRY(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
      PRNU_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
      PRNU_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    }
    PRNU_CUDA_TRY(cudaEventRecord(c->ev_fork, s));
    PRNU_CUDA_TRY(cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
    for (int i0 = 0, k = 0; i0 < n; i0 += wave, ++k) {
      PassArgs ak = a;
      ak.item0 = i0;
      ak.nitems = std::min(wave, n - i0);
      ak.nunits = ak.nitems / share;
      ak.spec = a.spec + (size_t)(k & 1) * wave * H * Wh;
      ak.stats = a.stats + (size_t)(k & 1) * wave * H;
      launch_fixed_wave(ak, *fs, tn.variant, (k & 1) ? c->aux : s, c->launches);
    }
    PRNU_CUDA_TRY(cudaEventRecord(c->ev_join, c->aux));
    PRNU_CUDA_TRY(cudaStreamWaitEvent(s, c->ev_join, 0));
    PRNU_CUDA_TRY(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  } else if (!naive) {
    for (int i0 = 0; i0 < n; i0 += wave) {
      a.item0 = i0;
      a.nitems = std::min(wave, n - i0);
      a.nunits = a.nitems / share;
      if (fs) {
        launch_fixed_wave(a, *fs, tn.variant, s, c->launches);
      } else {
        launch_row_forward(a, true, nullptr, nullptr, s, c->launches);
        launch_col(a, 0, nullptr, nullptr, nullptr, s, c->launches);
        launch_row_inverse(a, nullptr, s, c->launches);
        launch_finalize(a, s, c->launches);
      }
    }
    if (fs) PRNU_CUDA_TRY(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  } else {
    // plain per-candidate path through full-size intermediates
    PRNU_CHECK_ARG(call.rdtype == kF32, "the per-candidate path takes FP32 residuals");
    const int nblk = 256;
    const size_t xbytes = (size_t)H * W * sizeof(float);
    ensure_buf(c, c->ws_misc, 2 * xbytes + nblk * (sizeof(float) + sizeof(int) + sizeof(double)) + 1024);
    char* base = reinterpret_cast<char*>(c->ws_misc.p);
    float* X = reinterpret_cast<float*>(base);
    float* C = reinterpret_cast<float*>(base + xbytes);
    double* bsum = reinterpret_cast<double*>(base + 2 * xbytes);
    float* bmax = reinterpret_cast<float*>(bsum + nblk);
    int* barg = reinterpret_cast<int*>(bmax + nblk);
    PassArgs b = a;
    b.resid = X;
    b.rdtype = kF32;
    b.nitems = 1;
    for (int k = 0; k < n; ++k) {
      a.item0 = k;
      a.nitems = 1;
      b.item0 = k;
      launch_naive_warp(a, X, s, c->launches);
      launch_row_forward(b, false, nullptr, nullptr, s, c->launches);
      launch_col(b, 3, nullptr, nullptr, nullptr, s, c->launches);
      launch_col(b, 2, nullptr, nullptr, nullptr, s, c->launches);
      launch_col(b, 4, nullptr, nullptr, nullptr, s, c->launches);
      launch_row_inverse(b, C, s, c->launches);
      launch_naive_pce(C, H, W, a.items + k, a.fps, a.scale, a.results + k, bmax, barg, bsum, nblk, s,
                       c->launches);
    }
  }
  launch_argmax(a.results, a.items, reinterpret_cast<const int*>(c->ws_groups.p), ngroups, share, d_out, call.scale,
                H, W, s, c->launches);
  if (d_all) {
    PRNU_CUDA_TRY(cudaMemsetAsync(d_all, 0xff, sizeof(double) * (size_t)ngroups * call.cmax, s));
    launch_scatter_all(a.results, n, call.cmax, d_all, s, c->launches);
  }
  PRNU_CUDA_TRY(cudaEventRecord(c->last_done, s));
}

static bool is_device_pointer(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static std::shared_ptr<Fingerprint> find_fp(prnu_ctx* c, uint64_t h) {
  auto it = c->fps.find(h);
  if (it == c->fps.end()) throw Error{PRNU_ENOTFOUND, "unknown fingerprint handle " + std::to_string(h)};
  return it->second;
}

static int search_common(prnu_ctx* ctx, const void* d_resid, int dtype, const float* d_scale, int F, int H, int W,
                         const uint64_t* fp_handles, int P, const prnu_grid* grid, const prnu_window* windows,
                         prnu_result* out, double* d_all_pce, prnu_stream stream, bool naive) {
  return guarded([&] {
    PRNU_CHECK_ARG(ctx, "NULL context");
    PRNU_CHECK_ARG(F >= 0 && P >= 0, "F and P must be >= 0");
    if (F == 0 || P == 0) return;
    PRNU_CHECK_ARG(d_resid && fp_handles && grid && out, "NULL argument");
    PRNU_CHECK_ARG(dtype == kF32 || dtype == kF16 || dtype == kBF16, "unknown residual dtype");
    validate_shape(H, W);
    DeviceGuard dg(ctx->device);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    SearchCall call;
    call.resid = d_resid;
    call.rdtype = dtype;
    call.scale = d_scale;
    call.F = F;
    call.H = H;
    call.W = W;
    for (int p = 0; p < P; ++p) {
      auto f = find_fp(ctx, fp_handles[p]);
      PRNU_CHECK_ARG(f->H == H && f->W == W, "fingerprint size differs from the frames");
      call.fps.push_back(f);
    }
    build_items(*grid, windows, F, P, call, share_forward(ctx, H, W, P, naive));
    const bool dev_out = is_device_pointer(out);
    prnu_result* d_out = out;
    if (!dev_out) {
      ensure_buf(ctx, ctx->ws_out, sizeof(prnu_result) * (size_t)F * P);
      d_out = reinterpret_cast<prnu_result*>(ctx->ws_out.p);
    }
    enqueue_search(ctx, call, d_out, d_all_pce, naive, s);
    if (!dev_out) {
      PRNU_CUDA_TRY(cudaMemcpyAsync(out, d_out, sizeof(prnu_result) * (size_t)F * P, cudaMemcpyDeviceToHost, s));
      PRNU_CUDA_TRY(cudaStreamSynchronize(s));
      if (*ctx->h_err) report_device_abort(ctx, s, "a bounded device-side wait timed out; the results are invalid");
    }
  });
}

// One item per node of a (frame, fingerprint) pair's node grid lams x ths.
static void add_pair_items(SearchCall& call, int f, int p, int group, const std::vector<float>& lams,
                           const std::vector<float>& ths) {
  const int nb = (int)ths.size();
  for (int a = 0; a < (int)lams.size(); ++a) {
    const double L = (double)lams[a];
    PRNU_CHECK_ARG(L > 0 && std::isfinite(L), "correction scales must be positive");
    for (int b = 0; b < nb; ++b) {
      const double t = (double)ths[b] * 3.14159265358979323846 / 180.0;
      const double cs = cos(t), sn = sin(t);
      WorkItem it;
      it.frame = f;
      it.fp = p;
      it.cand = a * nb + b;
      it.group = group;
      it.a11 = (float)(cs / L);
      it.a12 = (float)(sn / L);
      it.a21 = (float)(-sn / L);
      it.a22 = (float)(cs / L);
      it.lam = lams[a];
      it.th_deg = ths[b];
      call.items.push_back(it);
    }
  }
}

// ---------------------------------------------------------------- the correction as a device-side loop

namespace {

constexpr int kCorrHalfLam = 5;   // lambda nodes either side of the estimate (11 in all)

// Iteration work list on the device: for every active (frame, fingerprint)
// pair, in pair order, the 11 x (2 hb + 1) nodes around its estimate (the
// same float nodes and warp coefficients as add_pair_items); the pairs'
// order (who), their group table and the one-graph search's run descriptor
// (its arg-max per pair into out).  One block.
__global__ void k_corr_gen(int G, int P, const int* __restrict__ active, const float* __restrict__ cl,
                           const float* __restrict__ ct, float sl, float st, int hb, WorkItem* __restrict__ items,
                           CandResult* results, int* __restrict__ group_start, int* __restrict__ who,
                           prnu_result* out, DevRun* run) {
  __shared__ int s_nact;
  const int nb = 2 * hb + 1, per = (2 * kCorrHalfLam + 1) * nb;
  if (threadIdx.x == 0) {
    int k = 0;
    for (int g = 0; g < G; ++g)
      if (active[g]) {
        who[k] = g;
        group_start[k] = k * per;
        ++k;
      }
    group_start[k] = k * per;
    s_nact = k;
    DevRun r{};
    r.items = items;
    r.results = results;
    r.groups = group_start;
    r.out = out;
    r.n = k * per;
    r.share = 1;
    r.ngroups = k;
    *run = r;
  }
  __syncthreads();
  const int n = s_nact * per;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int k = i / per, c = i - k * per, g = who[k];
    const int a = c / nb, b = c - a * nb;
    const float lam = (float)((double)cl[g] + (double)(a - kCorrHalfLam) * (double)sl);
    const float th = (float)((double)ct[g] + (double)(b - hb) * (double)st);
    const double L = (double)lam;
    const double t = (double)th * 3.14159265358979323846 / 180.0;
    double sn, cs;
    sincos(t, &sn, &cs);
    WorkItem it;
    it.frame = g / P;
    it.fp = g % P;
    it.cand = c;
    it.group = k;
    it.a11 = (float)(cs / L);
    it.a12 = (float)(sn / L);
    it.a21 = (float)(-sn / L);
    it.a22 = (float)(cs / L);
    it.lam = lam;
    it.th_deg = th;
    items[i] = it;
  }
}

// After the iteration's search: per active pair, the best result so far, and
// the next estimate, or the pair leaves the loop (its arg-max is the centre
// node, or it found none).
__global__ void k_corr_update(const DevRun* run, const int* __restrict__ who, const prnu_result* __restrict__ out,
                              int centre, prnu_result* __restrict__ best, int* __restrict__ have,
                              int* __restrict__ active, float* __restrict__ cl, float* __restrict__ ct,
                              int* __restrict__ runs) {
  const int nact = run->ngroups;
  for (int k = threadIdx.x; k < nact; k += blockDim.x) {
    const int g = who[k];
    const prnu_result r = out[k];
    ++runs[g];
    if (!have[g] || r.pce > best[g].pce) {
      best[g] = r;
      have[g] = 1;
    }
    if (r.cand_idx == centre || r.cand_idx < 0) {
      active[g] = 0;
    } else {
      cl[g] = r.lam;
      ct[g] = r.th_deg;
    }
  }
}

}  // namespace

// The correction with its loop on the device (prnu_tuning.persistent = 2 on a
// size with compile-time-planned kernels; false otherwise): per iteration a
// kernel writes the work list of the active pairs, one graph launch scores it
// (the wave loop over one run, its arg-max per pair in the completion
// kernel), and a kernel updates the estimates.  max_iter iterations are
// enqueued at once; an iteration with no active pair has no candidates and
// its launch ends at once.  One synchronisation, at the end.
static bool run_correction_device(prnu_ctx* c, const void* d_resid, int dtype, const float* d_scale, int F, int H,
                                  int W, const std::vector<std::shared_ptr<Fingerprint>>& fps,
                                  const std::vector<float>& cl, const std::vector<float>& ct, int max_iter,
                                  int th_half1, prnu_result* out, int* iters, cudaStream_t s) {
  const Tuning tn = tuning_for(c, H, W);
  if (tn.persistent != 2 || tn.variant < 0) return false;
  const FixedShape* fs = find_fixed(H, W);
  if (!fs || !fixed_supports(*fs, H, tn.ppb)) return false;
  const int P = (int)fps.size(), G = F * P, Wh = W / 2;
  const int hb1 = th_half1 ? th_half1 : 50;
  const size_t per_max = (size_t)(2 * kCorrHalfLam + 1) * (2 * std::max(hb1, kCorrHalfLam) + 1);
  const size_t nmax = (size_t)G * per_max;
  PRNU_CHECK_ARG(nmax < (size_t)INT_MAX, "too many correction nodes");
  const int wave = std::max(1, std::min(tn.wave, kLoopMaxWave));

  if (*c->h_err)
    report_device_abort(c, s, "a bounded device-side wait of an earlier call timed out; its results are invalid");
  PRNU_CUDA_TRY(cudaStreamWaitEvent(s, c->last_done, 0));
  for (auto& f : fps) PRNU_CUDA_TRY(cudaStreamWaitEvent(s, f->ready, 0));
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t o_ct = al(sizeof(float) * G), o_act = o_ct + al(sizeof(float) * G), o_have = o_act + al(sizeof(int) * G),
               o_runs = o_have + al(sizeof(int) * G), o_who = o_runs + al(sizeof(int) * G),
               o_best = o_who + al(sizeof(int) * G), corr_bytes = o_best + al(sizeof(prnu_result) * G);
  ensure_buf(c, c->ws_items, sizeof(WorkItem) * nmax);
  ensure_buf(c, c->ws_results, sizeof(CandResult) * nmax);
  ensure_buf(c, c->ws_groups, sizeof(int) * (G + 1));
  ensure_buf(c, c->ws_fpdesc, sizeof(FpDesc) * std::max(P, 1));
  ensure_buf(c, c->ws_spec, (size_t)wave * H * Wh * sizeof(float2));
  ensure_buf(c, c->ws_stats, (size_t)wave * H * sizeof(RowStat));
  ensure_buf(c, c->ws_out, sizeof(prnu_result) * G);
  ensure_buf(c, c->ws_corr, corr_bytes);
  const ResidLayout lay = padded_layout(H, W);
  const bool pairs = dtype != kF32;
  ensure_buf(c, c->ws_pad, (size_t)F * lay.fpitch * (dtype == kF32 || pairs ? 4 : 2));
  char* cb = reinterpret_cast<char*>(c->ws_corr.p);
  float* d_cl = reinterpret_cast<float*>(cb);
  float* d_ct = reinterpret_cast<float*>(cb + o_ct);
  int* d_act = reinterpret_cast<int*>(cb + o_act);
  int* d_have = reinterpret_cast<int*>(cb + o_have);
  int* d_runs = reinterpret_cast<int*>(cb + o_runs);
  int* d_who = reinterpret_cast<int*>(cb + o_who);
  prnu_result* d_best = reinterpret_cast<prnu_result*>(cb + o_best);
  std::vector<FpDesc> fd;
  for (auto& f : fps) fd.push_back(fp_desc(*f));
  const std::vector<int> ones(G, 1);
  Stager stg(c);
  stg.add(c->ws_fpdesc.p, fd.data(), fd.size());
  stg.add(d_cl, cl.data(), cl.size());
  stg.add(d_ct, ct.data(), ct.size());
  stg.add(d_act, ones.data(), ones.size());
  stg.flush(s);
  PRNU_CUDA_TRY(cudaMemsetAsync(d_have, 0, 2 * al(sizeof(int) * G), s));   // have, runs
  launch_pad_frames(d_resid, dtype, F, H, W, c->ws_pad.p, s, c->launches, pairs ? 1 : 0);

  auto& bl = c->batch_loops[std::make_tuple(H, W, pairs ? (dtype == kF16 ? (int)kF16P : (int)kBF16P) : dtype)];
  if (!bl) bl.reset(new BatchLoop(c));
  WaveLoopConfig g;
  g.fs = fs;
  g.variant = tn.variant;
  g.ppb = tn.ppb;
  g.col_log2 = tn.col_log2;
  g.H = H;
  g.W = W;
  g.rdtype = pairs ? (dtype == kF16 ? kF16P : kBF16P) : dtype;
  g.wave = wave;
  g.fp_f32 = std::any_of(fd.begin(), fd.end(), [](const FpDesc& d) { return d.dtype == kF32; }) ? 1 : 0;
  g.spec = reinterpret_cast<float2*>(c->ws_spec.p);
  g.stats = reinterpret_cast<RowStat*>(c->ws_stats.p);
  g.spec_slots = wave;
  g.resid = c->ws_pad.p;
  g.fps = reinterpret_cast<const FpDesc*>(c->ws_fpdesc.p);
  g.scale = d_scale;
  g.err = c->d_err;
  g.stall = c->debug_stall;
  for (int n = 1; n <= max_iter; ++n) {
    // float32 steps 0.01 * 10^-(n-1) and 0.1 * 10^-(n-1) degrees, as the host loop takes them
    const float sl = (float)(0.01 * std::pow(10.0, -(n - 1))), st = (float)(0.1 * std::pow(10.0, -(n - 1)));
    const int hb = n == 1 ? hb1 : kCorrHalfLam;
    k_corr_gen<<<1, 1024, 0, s>>>(G, P, d_act, d_cl, d_ct, sl, st, hb,
                                  reinterpret_cast<WorkItem*>(c->ws_items.p),
                                  reinterpret_cast<CandResult*>(c->ws_results.p),
                                  reinterpret_cast<int*>(c->ws_groups.p), d_who,
                                  reinterpret_cast<prnu_result*>(c->ws_out.p), bl->ring_entry());
    PRNU_CUDA_TRY(cudaGetLastError());
    bl->run_written(g, s);
    const int nb = 2 * hb + 1;
    k_corr_update<<<1, 256, 0, s>>>(bl->ring_entry(), d_who, reinterpret_cast<const prnu_result*>(c->ws_out.p),
                                    kCorrHalfLam * nb + hb, d_best, d_have, d_act, d_cl, d_ct, d_runs);
    PRNU_CUDA_TRY(cudaGetLastError());
    c->launches.n += 2;
  }
  std::vector<int> runs(G);
  PRNU_CUDA_TRY(cudaMemcpyAsync(out, d_best, sizeof(prnu_result) * G, cudaMemcpyDeviceToHost, s));
  PRNU_CUDA_TRY(cudaMemcpyAsync(runs.data(), d_runs, sizeof(int) * G, cudaMemcpyDeviceToHost, s));
  PRNU_CUDA_TRY(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  PRNU_CUDA_TRY(cudaEventRecord(c->last_done, s));
  PRNU_CUDA_TRY(cudaStreamSynchronize(s));
  if (*c->h_err) report_device_abort(c, s, "a bounded device-side wait timed out; the results are invalid");
  if (iters)
    for (int k = 0; k < G; ++k) iters[k] = runs[k];
  return true;
}

}  // namespace prnu

using namespace prnu;

extern "C" {

// The iterative correction of Sec. 3.2 (Eq. 8) for every (frame, fingerprint)
// pair g = f*P + p from the start estimate (cl[g], ct[g]): exhaustive search over
// the node grid around the current estimate, steps 0.01 * 10^-(n-1) in lambda and
// 0.1 * 10^-(n-1) degrees in theta, until the best node is the centre or after
// max_iter levels.  out[g] = the best node of all levels; iters[g] (optional) =
// the levels run.  Caller holds ctx->mu and the device.
static void run_correction(prnu_ctx* ctx, const void* d_resid, int dtype, const float* d_scale, int F, int H,
                           int W, const std::vector<std::shared_ptr<Fingerprint>>& fps, std::vector<float> cl,
                           std::vector<float> ct, int max_iter, int th_half1, prnu_result* out, int* iters,
                           cudaStream_t s) {
  if (run_correction_device(ctx, d_resid, dtype, d_scale, F, H, W, fps, cl, ct, max_iter, th_half1, out, iters, s))
    return;
  constexpr int kHalf = 5;
  const int P = (int)fps.size();
  const int hb1 = th_half1 ? th_half1 : 50;
  const int G = F * P;
  std::vector<prnu_result> best(G);
  std::vector<char> have(G, 0), active(G, 1);
  std::vector<int> run(G, 0);
  ensure_buf(ctx, ctx->ws_out, sizeof(prnu_result) * (size_t)G);
  prnu_result* d_out = reinterpret_cast<prnu_result*>(ctx->ws_out.p);
  std::vector<prnu_result> res;
  for (int n = 1; n <= max_iter; ++n) {
    // float32 steps 0.01 * 10^-(n-1) and 0.1 * 10^-(n-1) degrees
    const float sl = (float)(0.01 * std::pow(10.0, -(n - 1))), st = (float)(0.1 * std::pow(10.0, -(n - 1)));
    const int hb = n == 1 ? hb1 : kHalf;
    SearchCall call;
    call.resid = d_resid;
    call.rdtype = dtype;
    call.scale = d_scale;
    call.F = F;
    call.H = H;
    call.W = W;
    call.fps = fps;
    call.cmax = (2 * kHalf + 1) * (2 * hb + 1);
    std::vector<int> who;   // active pair of each group of this iteration
    for (int g = 0; g < G; ++g) {
      if (!active[g]) continue;
      std::vector<float> lams, ths;
      for (int a = -kHalf; a <= kHalf; ++a) lams.push_back((float)((double)cl[g] + (double)a * (double)sl));
      for (int b = -hb; b <= hb; ++b) ths.push_back((float)((double)ct[g] + (double)b * (double)st));
      call.group_start.push_back((int)call.items.size());
      add_pair_items(call, g / P, g % P, (int)who.size(), lams, ths);
      who.push_back(g);
    }
    if (who.empty()) break;
    call.group_start.push_back((int)call.items.size());
    enqueue_search(ctx, call, d_out, nullptr, false, s);
    res.resize(who.size());
    PRNU_CUDA_TRY(cudaMemcpyAsync(res.data(), d_out, sizeof(prnu_result) * who.size(), cudaMemcpyDeviceToHost, s));
    PRNU_CUDA_TRY(cudaStreamSynchronize(s));
    if (*ctx->h_err) report_device_abort(ctx, s, "a bounded device-side wait timed out; the results are invalid");
    const int nb = 2 * hb + 1, centre = kHalf * nb + hb;
    for (size_t k = 0; k < who.size(); ++k) {
      const int g = who[k];
      const prnu_result& r = res[k];
      ++run[g];
      if (!have[g] || r.pce > best[g].pce) {
        best[g] = r;
        have[g] = 1;
      }
      if (r.cand_idx == centre || r.cand_idx < 0) {
        active[g] = 0;   // the estimate did not change
      } else {
        cl[g] = r.lam;
        ct[g] = r.th_deg;
      }
    }
  }
  for (int g = 0; g < G; ++g) {
    out[g] = best[g];
    if (iters) iters[g] = run[g];
  }
}

int eis_correction(prnu_ctx* ctx, const void* d_resid, int dtype, const float* d_scale, int F, int H, int W,
                   const uint64_t* fp_handles, int P, const float* init_lam, const float* init_th, int max_iter,
                   int th_half1, prnu_result* out, int* iters, prnu_stream stream) {
  return guarded([&] {
    PRNU_CHECK_ARG(ctx, "NULL context");
    PRNU_CHECK_ARG(F >= 0 && P >= 0, "F and P must be >= 0");
    if (F == 0 || P == 0) return;
    PRNU_CHECK_ARG(d_resid && fp_handles && out, "NULL argument");
    PRNU_CHECK_ARG(dtype == kF32 || dtype == kF16 || dtype == kBF16, "unknown residual dtype");
    PRNU_CHECK_ARG(max_iter >= 1, "max_iter must be >= 1");
    PRNU_CHECK_ARG(th_half1 >= 0 && th_half1 <= 4096, "th_half1 must be in 0..4096");
    validate_shape(H, W);
    DeviceGuard dg(ctx->device);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int G = F * P;
    std::vector<std::shared_ptr<Fingerprint>> fps;
    for (int p = 0; p < P; ++p) {
      auto f = find_fp(ctx, fp_handles[p]);
      PRNU_CHECK_ARG(f->H == H && f->W == W, "fingerprint size differs from the frames");
      fps.push_back(f);
    }
    std::vector<float> cl(G), ct(G);
    for (int g = 0; g < G; ++g) {
      cl[g] = init_lam ? init_lam[g] : 1.0f;
      ct[g] = init_th ? init_th[g] : 0.0f;
      PRNU_CHECK_ARG(std::isfinite(cl[g]) && cl[g] > 0 && std::isfinite(ct[g]), "bad start estimate");
    }
    run_correction(ctx, d_resid, dtype, d_scale, F, H, W, fps, std::move(cl), std::move(ct), max_iter, th_half1,
                   out, iters, s);
  });
}

// (lambda, theta) of the similarity nearest to the linear part of a homography
static void similarity_of(const double* Hm, float* lam, float* th_deg) {
  for (int i = 0; i < 9; ++i) PRNU_CHECK_ARG(std::isfinite(Hm[i]), "non-finite homography entry");
  PRNU_CHECK_ARG(Hm[8] != 0.0, "homography with h33 = 0");
  // linear part M (x = column, y = row), projected on {[a, -b], [b, a]}:
  // a = lambda cos(theta), b = lambda sin(theta)
  const double m00 = Hm[0] / Hm[8], m01 = Hm[1] / Hm[8], m10 = Hm[3] / Hm[8], m11 = Hm[4] / Hm[8];
  const double a = 0.5 * (m00 + m11), b = 0.5 * (m10 - m01);
  const double L = std::hypot(a, b);
  PRNU_CHECK_ARG(L > 0 && std::isfinite(L), "homography without a similarity part");
  *lam = (float)L;
  *th_deg = (float)(std::atan2(b, a) * 180.0 / 3.14159265358979323846);
}

int similarity_from_homography(const double* Hm, float* lam, float* th_deg) {
  return guarded([&] {
    PRNU_CHECK_ARG(Hm && lam && th_deg, "NULL argument");
    similarity_of(Hm, lam, th_deg);
  });
}

int eis_invert_video(prnu_ctx* ctx, const void* d_resid, int dtype, const float* d_scale, int F, int H, int W,
                     uint64_t fp_handle, const double* homographies, int max_iter, int th_half1, double tau,
                     double* gamma, double* mean_gamma, int* decision, prnu_result* best, int* from_reg,
                     prnu_stream stream) {
  return guarded([&] {
    PRNU_CHECK_ARG(ctx, "NULL context");
    PRNU_CHECK_ARG(F >= 1, "F must be >= 1 (the anchor)");
    PRNU_CHECK_ARG(d_resid && gamma, "NULL argument");
    PRNU_CHECK_ARG(dtype == kF32 || dtype == kF16 || dtype == kBF16, "unknown residual dtype");
    PRNU_CHECK_ARG(max_iter >= 1, "max_iter must be >= 1");
    PRNU_CHECK_ARG(th_half1 >= 0 && th_half1 <= 4096, "th_half1 must be in 0..4096");
    PRNU_CHECK_ARG(std::isfinite(tau), "tau must be finite");
    validate_shape(H, W);
    DeviceGuard dg(ctx->device);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    auto f = find_fp(ctx, fp_handle);
    PRNU_CHECK_ARG(f->H == H && f->W == W, "fingerprint size differs from the frames");
    const std::vector<std::shared_ptr<Fingerprint>> fps{f};
    std::vector<float> cl(F, 1.0f), ct(F, 0.0f);
    std::vector<int> use(F, 0);
    if (homographies && F > 1) {
      // the co-registered frame against the frame itself: one single-node
      // group each, (lambda_v, theta_v) from H_v and the identity (1, 0)
      std::vector<float> rl(F), rt(F);
      for (int v = 1; v < F; ++v) similarity_of(homographies + 9 * (size_t)v, &rl[v], &rt[v]);
      SearchCall call;
      call.resid = d_resid;
      call.rdtype = dtype;
      call.scale = d_scale;
      call.F = F;
      call.H = H;
      call.W = W;
      call.fps = fps;
      call.cmax = 1;
      for (int v = 1; v < F; ++v) {
        for (int k = 0; k < 2; ++k) {
          const int grp = 2 * (v - 1) + k;
          call.group_start.push_back((int)call.items.size());
          add_pair_items(call, v, 0, grp, {k == 0 ? rl[v] : 1.0f}, {k == 0 ? rt[v] : 0.0f});
        }
      }
      call.group_start.push_back((int)call.items.size());
      const int ng = 2 * (F - 1);
      ensure_buf(ctx, ctx->ws_out, sizeof(prnu_result) * (size_t)ng);
      prnu_result* d_out = reinterpret_cast<prnu_result*>(ctx->ws_out.p);
      enqueue_search(ctx, call, d_out, nullptr, false, s);
      std::vector<prnu_result> res(ng);
      PRNU_CUDA_TRY(cudaMemcpyAsync(res.data(), d_out, sizeof(prnu_result) * ng, cudaMemcpyDeviceToHost, s));
      PRNU_CUDA_TRY(cudaStreamSynchronize(s));
      if (*ctx->h_err) report_device_abort(ctx, s, "a bounded device-side wait timed out; the results are invalid");
      for (int v = 1; v < F; ++v) {
        if (res[2 * (v - 1)].pce > res[2 * (v - 1) + 1].pce) {
          cl[v] = rl[v];
          ct[v] = rt[v];
          use[v] = 1;
        }
      }
    }
    std::vector<prnu_result> out(F);
    run_correction(ctx, d_resid, dtype, d_scale, F, H, W, fps, std::move(cl), std::move(ct), max_iter, th_half1,
                   out.data(), nullptr, s);
    double sum = 0.0;
    for (int v = 0; v < F; ++v) {
      gamma[v] = out[v].pce;
      sum += out[v].pce;
      if (best) best[v] = out[v];
      if (from_reg) from_reg[v] = use[v];
    }
    const double m = sum / (double)F;
    if (mean_gamma) *mean_gamma = m;
    if (decision) *decision = m > tau ? 1 : 0;
  });
}


const char* prnu_last_error(void) { return g_last_error.c_str(); }

uint64_t prnu_launch_count(const prnu_ctx* ctx) { return ctx ? ctx->launches.n.load() : 0; }

int prnu_create(prnu_ctx** out, int device, size_t hbm_budget_bytes) {
  return guarded([&] {
    PRNU_CHECK_ARG(out, "NULL out");
    int ndev = 0;
    PRNU_CUDA_TRY(cudaGetDeviceCount(&ndev));
    PRNU_CHECK_ARG(device >= 0 && device < ndev, "no such CUDA device");
    DeviceGuard dg(device);
    PRNU_CUDA_TRY(cudaSetDevice(device));
    std::unique_ptr<prnu_ctx> c(new prnu_ctx());
    c->device = device;
    PRNU_CUDA_TRY(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device));
    size_t fr = 0, tot = 0;
    PRNU_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    c->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)fr);
    // twiddles w_n^k = exp(-2 pi i k / n) for every 5-smooth n <= 4096
    c->tw_off.assign(kMaxFft + 1, -1);
    std::vector<float2> tw;
    for (int n = 1; n <= kMaxFft; ++n) {
      if (!is_5smooth(n)) continue;
      c->tw_off[n] = (int)tw.size();
      for (int k = 0; k < n; ++k) {
        const double a = 2.0 * 3.14159265358979323846 * (double)k / (double)n;
        tw.push_back(make_float2((float)cos(a), (float)(-sin(a))));
      }
    }
    const size_t twb = tw.size() * sizeof(float2);
    c->d_tw = reinterpret_cast<float2*>(ctx_alloc(c.get(), twb));
    c->tw_bytes = twb;
    PRNU_CUDA_TRY(cudaMemcpy(c->d_tw, tw.data(), twb, cudaMemcpyHostToDevice));
    PRNU_CUDA_TRY(cudaEventCreateWithFlags(&c->last_done, cudaEventDisableTiming));
    PRNU_CUDA_TRY(cudaEventCreateWithFlags(&c->stage_free, cudaEventDisableTiming));
    PRNU_CUDA_TRY(cudaEventRecord(c->last_done, 0));
    PRNU_CUDA_TRY(cudaEventRecord(c->stage_free, 0));
    PRNU_CUDA_TRY(cudaHostAlloc((void**)&c->h_err, sizeof(int), cudaHostAllocDefault));
    *c->h_err = 0;
    c->d_err = reinterpret_cast<int*>(ctx_alloc(c.get(), sizeof(int)));
    PRNU_CUDA_TRY(cudaMemset(c->d_err, 0, sizeof(int)));
    set_kernel_attributes();
    *out = c.release();
  });
}

int prnu_destroy(prnu_ctx* ctx) {
  if (!ctx) return PRNU_OK;
  return guarded([&] {
    DeviceGuard dg(ctx->device);
    ctx->server.reset();
    cudaDeviceSynchronize();
    ctx->batch_loops.clear();
    for (auto& kv : ctx->fps) {
      auto& f = kv.second;
      if (f->refs > 0 && f.use_count() == 1) {
        ctx_free(ctx, f->d_spec, f->bytes);
        ctx_free(ctx, f->d_scal, 3 * sizeof(float));
        cudaEventDestroy(f->ready);
      }
    }
    ctx->fps.clear();
    for (DeviceBuf* b : {&ctx->ws_spec, &ctx->ws_stats, &ctx->ws_items, &ctx->ws_results, &ctx->ws_groups,
                         &ctx->ws_out, &ctx->ws_fpdesc, &ctx->ws_misc, &ctx->ws_resid, &ctx->ws_persist, &ctx->ws_pad, &ctx->ws_fpest,
                         &ctx->ws_lit, &ctx->ws_litx, &ctx->ws_litpart, &ctx->ws_renders, &ctx->ws_resize,
                         &ctx->ws_wav, &ctx->ws_corr})
      ctx_free(ctx, b->p, b->bytes);
    ctx_free(ctx, ctx->d_tw, ctx->tw_bytes);
    ctx_free(ctx, ctx->d_err, sizeof(int));
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    if (ctx->h_err) cudaFreeHost(ctx->h_err);
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    cudaEventDestroy(ctx->last_done);
    cudaEventDestroy(ctx->stage_free);
    delete ctx;
  });
}

int prnu_residual(prnu_ctx* ctx, const uint8_t* d_frames, int F, int H, int W, size_t pitch, int flags, int out_dtype,
                  void* d_out, float* d_scale, prnu_stream stream) {
  return guarded([&] {
    PRNU_CHECK_ARG(ctx, "NULL context");
    PRNU_CHECK_ARG(F >= 0, "F must be >= 0");
    if (F == 0) return;
    PRNU_CHECK_ARG(d_frames && d_out, "NULL argument");
    PRNU_CHECK_ARG(H >= 1 && W >= 1 && (long long)H * W <= (1LL << 26), "bad frame size");
    if (pitch == 0) pitch = (size_t)W;
    PRNU_CHECK_ARG(pitch >= (size_t)W, "pitch < W");
    PRNU_CHECK_ARG(out_dtype == kF32 || out_dtype == kF16 || out_dtype == kBF16, "unknown output dtype");
    PRNU_CHECK_ARG((flags & ~(PRNU_WEIGHT_BY_INTENSITY | PRNU_NORMALISE)) == 0, "unknown flags");
    DeviceGuard dg(ctx->device);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    PRNU_CUDA_TRY(cudaStreamWaitEvent(s, ctx->last_done, 0));
    const size_t np = residual_partials_needed(F, H, W);
    const size_t need = sizeof(unsigned long long) * F + sizeof(double) * np + sizeof(float) * F + 512;
    ensure_buf(ctx, ctx->ws_resid, need);
    char* base = reinterpret_cast<char*>(ctx->ws_resid.p);
    auto* acc = reinterpret_cast<unsigned long long*>(base);
    auto* partials = reinterpret_cast<double*>(base + ((sizeof(unsigned long long) * F + 255) & ~(size_t)255));
    float* scale = d_scale;
    if (!scale && (flags & PRNU_NORMALISE))
      scale = reinterpret_cast<float*>(reinterpret_cast<char*>(partials) + ((sizeof(double) * np + 255) & ~(size_t)255));
    launch_residual(d_frames, F, H, W, pitch, flags, out_dtype, d_out, scale, acc, partials, (int)np, s,
                    ctx->launches);
    PRNU_CUDA_TRY(cudaEventRecord(ctx->last_done, s));
  });
}

int prnu_residual_wavelet(prnu_ctx* ctx, const uint8_t* d_frames, int F, int H, int W, size_t pitch, int flags,
                          int out_dtype, double sigma0, void* d_out, float* d_scale, prnu_stream stream) {
  return guarded([&] {
    PRNU_CHECK_ARG(ctx, "NULL context");
    PRNU_CHECK_ARG(F >= 0, "F must be >= 0");
    if (F == 0) return;
    PRNU_CHECK_ARG(d_frames && d_out, "NULL argument");
    PRNU_CHECK_ARG(H >= 16 && W >= 16 && (long long)H * W <= (1LL << 26), "frames must be at least 16 x 16");
    if (pitch == 0) pitch = (size_t)W;
    PRNU_CHECK_ARG(pitch >= (size_t)W, "pitch < W");
    PRNU_CHECK_ARG(out_dtype == kF32 || out_dtype == kF16 || out_dtype == kBF16, "unknown output dtype");
    PRNU_CHECK_ARG((flags & ~(PRNU_WEIGHT_BY_INTENSITY | PRNU_NORMALISE)) == 0, "unknown flags");
    PRNU_CHECK_ARG(std::isfinite(sigma0) && sigma0 >= 0.0, "sigma0 must be finite and >= 0");
    DeviceGuard dg(ctx->device);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    PRNU_CUDA_TRY(cudaStreamWaitEvent(s, ctx->last_done, 0));
    const size_t Hp = (H + 15) / 16 * 16, Wp = (W + 15) / 16 * 16;
    // up to 16 frames at a time, within a quarter of what the budget leaves
    const size_t used = ctx->used.load(), avail = ctx->budget > used ? ctx->budget - used : 0;
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>({(size_t)F, 16, avail / 4 / (2 * Hp * Wp * 4)}));
    const size_t buf = Hp * Wp * chunk * sizeof(float);
    const size_t np = (flags & PRNU_NORMALISE) ? wavelet_partials_needed(F, H, W) : 0;
    const size_t sc = (flags & PRNU_NORMALISE) && !d_scale ? sizeof(float) * F : 0;
    ensure_buf(ctx, ctx->ws_wav, 2 * buf + sizeof(double) * np + sc + 1024);
    char* base = reinterpret_cast<char*>(ctx->ws_wav.p);
    float* bufA = reinterpret_cast<float*>(base);
    float* bufT = reinterpret_cast<float*>(base + buf);
    double* partials = reinterpret_cast<double*>(base + 2 * buf);
    float* scale = d_scale ? d_scale : (sc ? reinterpret_cast<float*>(base + 2 * buf + sizeof(double) * np) : nullptr);
    launch_wavelet_residual(d_frames, F, H, W, pitch, flags, out_dtype, (float)sigma0, d_out, scale, bufA, bufT, chunk,
                            partials, s, ctx->launches);
    PRNU_CUDA_TRY(cudaEventRecord(ctx->last_done, s));
  });
}

int prnu_fingerprint_estimate(prnu_ctx* ctx, const uint8_t* d_frames, int L, int H, int W, size_t pitch, float* d_K,
                              prnu_stream stream) {
  return guarded([&] {
    PRNU_CHECK_ARG(ctx && d_frames && d_K, "NULL argument");
    PRNU_CHECK_ARG(L >= 1, "L must be >= 1");
    PRNU_CHECK_ARG(H >= 1 && W >= 1 && (long long)H * W <= (1LL << 26), "bad frame size");
    if (pitch == 0) pitch = (size_t)W;
    PRNU_CHECK_ARG(pitch >= (size_t)W, "pitch < W");
    DeviceGuard dg(ctx->device);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    PRNU_CUDA_TRY(cudaStreamWaitEvent(s, ctx->last_done, 0));
    constexpr int kChunk = 16;
    const size_t n = (size_t)H * W;
    const int C0 = std::min(L, kChunk);
    const size_t rb = (sizeof(float) * n * C0 + 255) / 256 * 256, db = (sizeof(double) * n + 255) / 256 * 256;
    ensure_buf(ctx, ctx->ws_fpest, rb + 2 * db);
    char* base = reinterpret_cast<char*>(ctx->ws_fpest.p);
    float* R = reinterpret_cast<float*>(base);
    double* num = reinterpret_cast<double*>(base + rb);
    double* den = reinterpret_cast<double*>(base + rb + db);
    const size_t np = residual_partials_needed(C0, H, W);
    ensure_buf(ctx, ctx->ws_resid, sizeof(unsigned long long) * C0 + 256 + sizeof(double) * np);
    auto* acc = reinterpret_cast<unsigned long long*>(ctx->ws_resid.p);
    auto* partials = reinterpret_cast<double*>(reinterpret_cast<char*>(ctx->ws_resid.p) +
                                               ((sizeof(unsigned long long) * C0 + 255) & ~(size_t)255));
    for (int l0 = 0; l0 < L; l0 += kChunk) {
      const int Lc = std::min(kChunk, L - l0);
      const uint8_t* fr = d_frames + (size_t)l0 * H * pitch;
      launch_residual(fr, Lc, H, W, pitch, PRNU_WEIGHT_BY_INTENSITY, kF32, R, nullptr, acc, partials,
                      (int)residual_partials_needed(Lc, H, W), s, ctx->launches);
      launch_fp_estimate_accumulate(R, fr, pitch, Lc, H, W, num, den, l0 == 0, s, ctx->launches);
    }
    launch_fp_estimate_divide(num, den, d_K, n, s, ctx->launches);
    PRNU_CUDA_TRY(cudaEventRecord(ctx->last_done, s));
  });
}

int prnu_fingerprint_term(prnu_ctx* ctx, const float* d_K, int H, int W, int store_dtype, uint64_t* out_handle,
                          prnu_stream stream) {
  return guarded([&] {
    PRNU_CHECK_ARG(ctx && d_K && out_handle, "NULL argument");
    validate_shape(H, W);
    PRNU_CHECK_ARG(store_dtype == kF32 || store_dtype == kF16 || store_dtype == kBF16, "unknown storage dtype");
    DeviceGuard dg(ctx->device);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int Wh = W / 2;
    const bool half = store_dtype != kF32;
    auto f = std::make_shared<Fingerprint>();
    f->H = H;
    f->W = W;
    f->dtype = half ? kF16 : kF32;
    f->bytes = (size_t)H * Wh * (half ? sizeof(__half2) : sizeof(float2));
    // the column pass of the compile-time-planned kernels reads strips of the
    // spectrum by TMA: its descriptors live right after the spectrum
    alignas(64) unsigned char tmaps[kFpTmapBytes];
    const size_t tmap_off = (f->bytes + 127) / 128 * 128;
    f->bytes = tmap_off + kFpTmapBytes;
    f->d_spec = ctx_alloc(ctx, f->bytes);
    try {
      if (encode_fp_tmaps(f->d_spec, f->dtype, H, W, tmaps)) {
        PRNU_CUDA_TRY(
            cudaMemcpy(static_cast<char*>(f->d_spec) + tmap_off, tmaps, kFpTmapBytes, cudaMemcpyHostToDevice));
        f->tmap_off = tmap_off;
      }
      f->d_scal = reinterpret_cast<float*>(ctx_alloc(ctx, 3 * sizeof(float)));
    } catch (...) {
      ctx_free(ctx, f->d_spec, f->bytes);
      throw;
    }
    PRNU_CUDA_TRY(cudaEventCreateWithFlags(&f->ready, cudaEventDisableTiming));
    PRNU_CUDA_TRY(cudaStreamWaitEvent(s, ctx->last_done, 0));
    const int nblk = 256;
    ensure_buf(ctx, ctx->ws_misc, 2 * nblk * sizeof(double));
    ensure_buf(ctx, ctx->ws_spec, (size_t)H * Wh * sizeof(float2));
    const FftPlan prow = make_plan(W, ctx->tw_off), pcol = make_plan(H, ctx->tw_off);
    int rowT, rowMB;
    row_launch_shape(prow, &rowT, &rowMB);
    Tuning tn = tuning_for(ctx, H, W);
    launch_fp_stats(d_K, H, W, reinterpret_cast<double*>(ctx->ws_misc.p), nblk, f->d_scal, f->d_scal + 1,
                    f->d_scal + 2, half, s, ctx->launches);
    PassArgs a{};
    a.resid = d_K;
    a.rdtype = kF32;
    a.H = H;
    a.W = W;
    a.item0 = 0;
    a.nitems = 1;
    a.spec = reinterpret_cast<float2*>(ctx->ws_spec.p);
    a.tw = ctx->d_tw;
    a.prow = prow;
    a.pcol = pcol;
    a.pairs_per_block = tn.ppb;
    a.col_log2 = tn.col_log2;
    a.row_threads = rowT;
    launch_row_forward(a, false, f->d_scal, nullptr, s, ctx->launches);
    launch_col(a, 1, half ? nullptr : reinterpret_cast<float2*>(f->d_spec), half ? f->d_spec : nullptr,
               f->d_scal + 1, s, ctx->launches);
    PRNU_CUDA_TRY(cudaEventRecord(f->ready, s));
    PRNU_CUDA_TRY(cudaEventRecord(ctx->last_done, s));
    f->refs = 1;
    const uint64_t h = ctx->next_handle++;
    ctx->fps[h] = f;
    *out_handle = h;
  });
}

int prnu_fingerprint_release(prnu_ctx* ctx, uint64_t handle) {
  return guarded([&] {
    PRNU_CHECK_ARG(ctx, "NULL context");
    DeviceGuard dg(ctx->device);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    auto it = ctx->fps.find(handle);
    if (it == ctx->fps.end()) throw Error{PRNU_ENOTFOUND, "unknown fingerprint handle"};
    auto f = it->second;
    ctx->fps.erase(it);
    // freed once no call or query holds it; pending work is ordered by last_done
    if (f.use_count() == 1) {
      PRNU_CUDA_TRY(cudaEventSynchronize(ctx->last_done));
      ctx_free(ctx, f->d_spec, f->bytes);
      ctx_free(ctx, f->d_scal, 3 * sizeof(float));
      cudaEventDestroy(f->ready);
      f->d_spec = nullptr;
      f->d_scal = nullptr;
    }
  });
}

int eis_grid_search(prnu_ctx* ctx, const void* d_resid, int dtype, const float* d_scale, int F, int H, int W,
                    const uint64_t* fp_handles, int P, const prnu_grid* grid, const prnu_window* windows,
                    prnu_result* out, double* d_all_pce, prnu_stream stream) {
  return search_common(ctx, d_resid, dtype, d_scale, F, H, W, fp_handles, P, grid, windows, out, d_all_pce, stream,
                       false);
}

int eis_grid_search_naive(prnu_ctx* ctx, const void* d_resid, int dtype, const float* d_scale, int F, int H, int W,
                          const uint64_t* fp_handles, int P, const prnu_grid* grid, const prnu_window* windows,
                          prnu_result* out, double* d_all_pce, prnu_stream stream) {
  return search_common(ctx, d_resid, dtype, d_scale, F, H, W, fp_handles, P, grid, windows, out, d_all_pce, stream,
                       true);
}

// The frame-literal search of Sec. 3.2: per candidate the frame is warped and
// its residual extracted (launch_literal_residuals, into the zero-bordered
// layout), then the search runs on those residuals with the identity warp.
// Candidates are rendered in chunks of at most kLitChunkBytes of residuals;
// every fingerprint of a frame searches the same renders.  The best per
// (frame, fingerprint) is kept over the chunks on the host: a higher PCE
// replaces it, so ties keep the lowest candidate index.
static constexpr size_t kLitChunkBytes = (size_t)2 << 30;   // and as much again for the warped frames

int eis_grid_search_frames(prnu_ctx* ctx, const uint8_t* d_frames, int F, int H, int W, size_t pitch, int flags,
                           const uint64_t* fp_handles, int P, const prnu_grid* grid, const prnu_window* windows,
                           prnu_result* out, prnu_stream stream) {
  return guarded([&] {
    PRNU_CHECK_ARG(ctx, "NULL context");
    PRNU_CHECK_ARG(F >= 0 && P >= 0, "F and P must be >= 0");
    if (F == 0 || P == 0) return;
    PRNU_CHECK_ARG(d_frames && fp_handles && grid && out, "NULL argument");
    PRNU_CHECK_ARG((flags & ~PRNU_WEIGHT_BY_INTENSITY) == 0, "flags: only PRNU_WEIGHT_BY_INTENSITY applies");
    validate_shape(H, W);
    if (pitch == 0) pitch = (size_t)W;
    PRNU_CHECK_ARG(pitch >= (size_t)W, "pitch must be >= W");
    PRNU_CHECK_ARG(pitch * (size_t)H <= (size_t)INT_MAX, "a frame must span at most 2^31 - 1 bytes");
    DeviceGuard dg(ctx->device);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<std::shared_ptr<Fingerprint>> fps;
    for (int p = 0; p < P; ++p) {
      auto f = find_fp(ctx, fp_handles[p]);
      PRNU_CHECK_ARG(f->H == H && f->W == W, "fingerprint size differs from the frames");
      fps.push_back(f);
    }
    SearchCall all;
    build_items(*grid, windows, F, P, all);
    // renders: the candidates of fingerprint 0 of each frame (every fingerprint
    // of a frame has the same window)
    std::vector<WorkItem> renders;
    std::vector<int> render0(F + 1, 0);
    for (int f = 0; f < F; ++f) {
      render0[f] = (int)renders.size();
      for (int i = all.group_start[(size_t)f * P]; i < all.group_start[(size_t)f * P + 1]; ++i)
        renders.push_back(all.items[i]);
    }
    render0[F] = (int)renders.size();
    const ResidLayout lay = padded_layout(H, W);
    const size_t per = lay.fpitch * sizeof(float);
    // residuals and warped frames of a chunk: at most a quarter each of what the budget leaves
    const size_t used = ctx->used.load(), avail = ctx->budget > used ? ctx->budget - used : 0;
    const size_t cap = std::min(kLitChunkBytes, avail / 4);
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>(cap / per, renders.size()));
    ensure_buf(ctx, ctx->ws_lit, per * (size_t)chunk);
    ensure_buf(ctx, ctx->ws_litx, sizeof(float) * (size_t)H * W * chunk);
    ensure_buf(ctx, ctx->ws_litpart, sizeof(double) * (literal_partials_needed(chunk, H, W) + (size_t)chunk));
    ensure_buf(ctx, ctx->ws_renders, sizeof(WorkItem) * (size_t)chunk);
    float* d_lit = reinterpret_cast<float*>(ctx->ws_lit.p);
    double* d_part = reinterpret_cast<double*>(ctx->ws_litpart.p);
    float* d_nu2 = reinterpret_cast<float*>(d_part + literal_partials_needed(chunk, H, W));
    PRNU_CUDA_TRY(cudaStreamWaitEvent(s, ctx->last_done, 0));
    PRNU_CUDA_TRY(cudaMemsetAsync(d_lit, 0, per * (size_t)chunk, s));   // the zero border, never written after
    std::vector<prnu_result> best((size_t)F * P);
    std::vector<char> have((size_t)F * P, 0);
    std::vector<prnu_result> res;
    const int weight = (flags & PRNU_WEIGHT_BY_INTENSITY) ? 1 : 0;
    for (int r0 = 0; r0 < (int)renders.size(); r0 += chunk) {
      const int r1 = std::min<int>((int)renders.size(), r0 + chunk);
      {
        Stager st(ctx);
        st.add(ctx->ws_renders.p, renders.data() + r0, (size_t)(r1 - r0));
        st.flush(s);
      }
      launch_literal_residuals(d_frames, pitch, H, W, reinterpret_cast<const WorkItem*>(ctx->ws_renders.p), r1 - r0,
                               weight, d_lit, lay, reinterpret_cast<float*>(ctx->ws_litx.p), d_part, d_nu2, s,
                               ctx->launches);
      SearchCall call;
      call.resid = d_lit;
      call.rdtype = kF32;
      call.scale = nullptr;
      call.F = r1 - r0;
      call.H = H;
      call.W = W;
      call.fps = fps;
      call.cmax = all.cmax;
      call.prepadded = true;
      std::vector<int> gid;   // (frame, fingerprint) pair of each local group
      for (int f = 0; f < F; ++f) {
        const int a = std::max(r0, render0[f]), b = std::min(r1, render0[f + 1]);
        if (a >= b) continue;
        for (int p = 0; p < P; ++p) {
          call.group_start.push_back((int)call.items.size());
          for (int r = a; r < b; ++r) {
            WorkItem it = renders[r];
            it.frame = r - r0;
            it.fp = p;
            it.group = (int)gid.size();
            it.a11 = it.a22 = 1.f;
            it.a12 = it.a21 = 0.f;
            call.items.push_back(it);
          }
          gid.push_back(f * P + p);
        }
      }
      call.group_start.push_back((int)call.items.size());
      ensure_buf(ctx, ctx->ws_out, sizeof(prnu_result) * gid.size());
      prnu_result* d_out = reinterpret_cast<prnu_result*>(ctx->ws_out.p);
      enqueue_search(ctx, call, d_out, nullptr, false, s);
      res.resize(gid.size());
      PRNU_CUDA_TRY(cudaMemcpyAsync(res.data(), d_out, sizeof(prnu_result) * gid.size(), cudaMemcpyDeviceToHost, s));
      PRNU_CUDA_TRY(cudaStreamSynchronize(s));
      if (*ctx->h_err) report_device_abort(ctx, s, "a bounded device-side wait timed out; the results are invalid");
      for (size_t k = 0; k < gid.size(); ++k) {
        const int g = gid[k];
        if (!have[g] || res[k].pce > best[g].pce) {
          best[g] = res[k];
          have[g] = 1;
        }
      }
    }
    if (is_device_pointer(out)) {
      PRNU_CUDA_TRY(cudaMemcpyAsync(out, best.data(), sizeof(prnu_result) * best.size(), cudaMemcpyHostToDevice, s));
      PRNU_CUDA_TRY(cudaStreamSynchronize(s));
    } else {
      std::copy(best.begin(), best.end(), out);
    }
  });
}

// Taps of output samples first .. first + n - 1 of a length-n_in axis resized
// by `scale`: sample o at input position u = (o + 0.5) / scale - 0.5, tent
// weights max(0, 1 - |j - u| a) with a = min(scale, 1), indices clamped to the
// axis, normalised; T taps per sample (zero weight beyond its support).
static void resize_taps(int n_in, double scale, int first, int n, int T, std::vector<float>& w, std::vector<int>& idx) {
  const double a = std::min(scale, 1.0);
  w.assign((size_t)n * T, 0.f);
  idx.assign((size_t)n * T, 0);
  for (int o = 0; o < n; ++o) {
    const double u = ((double)(first + o) + 0.5) / scale - 0.5;
    const int lo = (int)std::floor(u - 1.0 / a);
    std::vector<double> ws;
    std::vector<int> js;
    double tot = 0.0;
    for (int j = lo; j <= lo + T - 1; ++j) {
      const double t = 1.0 - std::fabs((double)j - u) * a;
      if (t <= 0.0) continue;
      const int jj = std::min(std::max(j, 0), n_in - 1);
      ws.push_back(t);
      js.push_back(jj);
      tot += t;
    }
    for (size_t k = 0; k < ws.size(); ++k) {
      w[(size_t)o * T + k] = (float)(ws[k] / tot);
      idx[(size_t)o * T + k] = js[k];
    }
  }
}

int prnu_fingerprint_resize(prnu_ctx* ctx, const float* d_Kin, int Hin, int Win, size_t in_pitch, double scale,
                            int y0, int x0, float* d_Kout, int H, int W, prnu_stream stream) {
  return guarded([&] {
    PRNU_CHECK_ARG(ctx && d_Kin && d_Kout, "NULL argument");
    PRNU_CHECK_ARG(Hin >= 1 && Win >= 1 && H >= 1 && W >= 1, "sizes must be >= 1");
    PRNU_CHECK_ARG(std::isfinite(scale) && scale >= 1.0 / 64 && scale <= 64.0, "scale must be in [1/64, 64]");
    if (in_pitch == 0) in_pitch = (size_t)Win;
    PRNU_CHECK_ARG(in_pitch >= (size_t)Win, "in_pitch must be >= Win");
    const long long Hs = std::llround((double)Hin * scale), Ws = std::llround((double)Win * scale);
    PRNU_CHECK_ARG(y0 >= 0 && x0 >= 0 && y0 + (long long)H <= Hs && x0 + (long long)W <= Ws,
                   "the crop must lie inside the resized fingerprint");
    DeviceGuard dg(ctx->device);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // taps per sample: the tent spans (u - 1/a, u + 1/a), at most floor(2/a) + 2 integers
    const int T = (int)std::floor(2.0 / std::min(scale, 1.0)) + 2;
    std::vector<float> wy, wx;
    std::vector<int> iy, ix;
    resize_taps(Hin, scale, y0, H, T, wy, iy);
    resize_taps(Win, scale, x0, W, T, wx, ix);
    const size_t nwy = wy.size(), nwx = wx.size();
    ensure_buf(ctx, ctx->ws_resize, (nwy + nwx) * (sizeof(float) + sizeof(int)) + 1024);
    char* base = reinterpret_cast<char*>(ctx->ws_resize.p);
    float* d_wy = reinterpret_cast<float*>(base);
    float* d_wx = d_wy + nwy;
    int* d_iy = reinterpret_cast<int*>(d_wx + nwx);
    int* d_ix = d_iy + nwy;
    PRNU_CUDA_TRY(cudaStreamWaitEvent(s, ctx->last_done, 0));
    Stager st(ctx);
    st.add(d_wy, wy.data(), nwy);
    st.add(d_wx, wx.data(), nwx);
    st.add(d_iy, iy.data(), nwy);
    st.add(d_ix, ix.data(), nwx);
    st.flush(s);
    launch_fp_resize(d_Kin, in_pitch, d_wy, d_iy, d_wx, d_ix, T, H, W, d_Kout, s, ctx->launches);
    PRNU_CUDA_TRY(cudaEventRecord(ctx->last_done, s));
    PRNU_CUDA_TRY(cudaStreamSynchronize(s));
  });
}

int pce_score(prnu_ctx* ctx, const float* d_X, uint64_t fp_handle, int H, int W, double* pce, int* dy, int* dx,
              float* peak, prnu_stream stream) {
  return guarded([&] {
    PRNU_CHECK_ARG(ctx && d_X, "NULL argument");
    validate_shape(H, W);
    DeviceGuard dg(ctx->device);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    auto f = find_fp(ctx, fp_handle);
    PRNU_CHECK_ARG(f->H == H && f->W == W, "fingerprint size differs");
    const int Wh = W / 2;
    PRNU_CUDA_TRY(cudaStreamWaitEvent(s, ctx->last_done, 0));
    PRNU_CUDA_TRY(cudaStreamWaitEvent(s, f->ready, 0));
    ensure_buf(ctx, ctx->ws_items, sizeof(WorkItem));
    ensure_buf(ctx, ctx->ws_results, sizeof(CandResult));
    ensure_buf(ctx, ctx->ws_fpdesc, sizeof(FpDesc));
    ensure_buf(ctx, ctx->ws_spec, (size_t)H * Wh * sizeof(float2));
    ensure_buf(ctx, ctx->ws_stats, (size_t)H * sizeof(RowStat));
    WorkItem it{};
    it.a11 = it.a22 = 1.f;
    it.lam = 1.f;
    FpDesc fd{f->d_spec, f->dtype, f->d_scal + 2};
    Stager st(ctx);
    st.add(ctx->ws_items.p, &it, 1);
    st.add(ctx->ws_fpdesc.p, &fd, 1);
    st.flush(s);
    const FftPlan prow = make_plan(W, ctx->tw_off), pcol = make_plan(H, ctx->tw_off);
    int rowT, rowMB;
    row_launch_shape(prow, &rowT, &rowMB);
    Tuning tn = tuning_for(ctx, H, W);
    PassArgs a{};
    a.resid = d_X;
    a.rdtype = kF32;
    a.H = H;
    a.W = W;
    a.items = reinterpret_cast<const WorkItem*>(ctx->ws_items.p);
    a.item0 = 0;
    a.nitems = 1;
    a.spec = reinterpret_cast<float2*>(ctx->ws_spec.p);
    a.stats = reinterpret_cast<RowStat*>(ctx->ws_stats.p);
    a.results = reinterpret_cast<CandResult*>(ctx->ws_results.p);
    a.fps = reinterpret_cast<const FpDesc*>(ctx->ws_fpdesc.p);
    a.tw = ctx->d_tw;
    a.prow = prow;
    a.pcol = pcol;
    a.pairs_per_block = tn.ppb;
    a.col_log2 = tn.col_log2;
    a.row_threads = rowT;
    launch_row_forward(a, false, nullptr, nullptr, s, ctx->launches);
    launch_col(a, 0, nullptr, nullptr, nullptr, s, ctx->launches);
    launch_row_inverse(a, nullptr, s, ctx->launches);
    launch_finalize(a, s, ctx->launches);
    CandResult r{};
    PRNU_CUDA_TRY(cudaMemcpyAsync(&r, a.results, sizeof(CandResult), cudaMemcpyDeviceToHost, s));
    PRNU_CUDA_TRY(cudaEventRecord(ctx->last_done, s));
    PRNU_CUDA_TRY(cudaStreamSynchronize(s));
    if (pce) *pce = r.pce;
    if (dy) *dy = r.py < H / 2 ? r.py : r.py - H;
    if (dx) *dx = r.px < W / 2 ? r.px : r.px - W;
    if (peak) *peak = r.peak;
  });
}

int prnu_profile_begin(prnu_ctx* ctx) {
  return guarded([&] {
    PRNU_CHECK_ARG(ctx, "NULL context");
    DeviceGuard dg(ctx->device);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    auto& lc = ctx->launches;
    std::lock_guard<std::mutex> lk2(lc.mu);
    for (auto& r : lc.recs) {
      lc.pool.push_back(r.a);
      lc.pool.push_back(r.b);
    }
    lc.recs.clear();
    lc.profiling = true;
  });
}

int prnu_profile_end(prnu_ctx* ctx, prnu_kernel_stat* out, int max, int* n_out) {
  return guarded([&] {
    PRNU_CHECK_ARG(ctx && out && max >= 1, "bad arguments");
    DeviceGuard dg(ctx->device);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    auto& lc = ctx->launches;
    std::lock_guard<std::mutex> lk2(lc.mu);
    lc.profiling = false;
    std::vector<uint64_t> cnt(kKindCount, 0);
    std::vector<double> ms(kKindCount, 0.0);
    for (auto& r : lc.recs) {
      PRNU_CUDA_TRY(cudaEventSynchronize(r.b));
      float t = 0.f;
      PRNU_CUDA_TRY(cudaEventElapsedTime(&t, r.a, r.b));
      cnt[r.kind]++;
      ms[r.kind] += t;
      lc.pool.push_back(r.a);
      lc.pool.push_back(r.b);
    }
    lc.recs.clear();
    int k = 0;
    for (int i = 0; i < kKindCount; ++i) {
      if (!cnt[i]) continue;
      if (k < max) {
        memset(out[k].name, 0, sizeof(out[k].name));
        strncpy(out[k].name, kKindNames[i], sizeof(out[k].name) - 1);
        out[k].launches = cnt[i];
        out[k].total_ms = ms[i];
      }
      ++k;
    }
    if (n_out) *n_out = k;
  });
}

int prnu_get_tuning(prnu_ctx* ctx, int H, int W, prnu_tuning* out) {
  return guarded([&] {
    PRNU_CHECK_ARG(ctx && out, "NULL argument");
    validate_shape(H, W);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    Tuning t = tuning_for(ctx, H, W);
    out->col_width = 1 << t.col_log2;
    out->pairs_per_block = t.ppb;
    out->wave = t.wave;
    out->variant = t.variant;
    out->persistent = t.persistent;
    out->streams = t.streams;
    out->share_forward = t.share;
  });
}

int prnu_debug_set(prnu_ctx* ctx, int key, int value) {
  return guarded([&] {
    PRNU_CHECK_ARG(ctx, "NULL context");
    PRNU_CHECK_ARG(key == PRNU_DEBUG_STALL_DEVICE_WAITS, "unknown debug key");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    ctx->debug_stall = value ? 1 : 0;
  });
}

int prnu_set_tuning(prnu_ctx* ctx, int H, int W, const prnu_tuning* cfg) {
  return guarded([&] {
    PRNU_CHECK_ARG(ctx && cfg, "NULL argument");
    validate_shape(H, W);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    int lg = -1;
    for (int k = 0; k <= 4; ++k)
      if (cfg->col_width == (1 << k)) lg = k;
    PRNU_CHECK_ARG(lg >= 0, "col_width must be 1, 2, 4, 8 or 16");
    PRNU_CHECK_ARG(cfg->pairs_per_block == 1 || cfg->pairs_per_block == 2 || cfg->pairs_per_block == 4,
                   "pairs_per_block must be 1, 2 or 4");
    PRNU_CHECK_ARG(cfg->wave >= 1, "wave must be >= 1");
    FftPlan pc = make_plan(H, ctx->tw_off), pr = make_plan(W, ctx->tw_off);
    int T, mb;
    col_launch_shape(pc, lg, &T, &mb);
    PRNU_CHECK_ARG(2 * (size_t)H * (1u << lg) * sizeof(float2) <= 227 * 1024, "column strip exceeds shared memory");
    row_launch_shape(pr, &T, &mb);
    PRNU_CHECK_ARG(T * cfg->pairs_per_block <= 512, "row block exceeds 512 threads");
    const FixedShape* fs = find_fixed(H, W);
    PRNU_CHECK_ARG(cfg->variant >= -1 && cfg->variant < (fs ? (int)fs->cols.size() : 0),
                   "variant out of range for this frame size (-1 = generic kernels)");
    PRNU_CHECK_ARG(cfg->persistent >= 0 && cfg->persistent <= 2, "persistent must be 0, 1 or 2");
    PRNU_CHECK_ARG(cfg->streams >= 0 && cfg->streams <= 2, "streams must be 0, 1 or 2");
    PRNU_CHECK_ARG(cfg->share_forward == 0 || cfg->share_forward == 1, "share_forward must be 0 or 1");
    ctx->tuning[{H, W}] = Tuning{lg, cfg->pairs_per_block, cfg->wave, cfg->variant, cfg->persistent,
                                 cfg->streams == 2 ? 2 : 1, cfg->share_forward};
  });
}

}  // extern "C"
