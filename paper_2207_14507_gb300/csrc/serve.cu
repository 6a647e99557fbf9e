// serve.cu -- continuous-batching query server behind query_submit / query_poll.
//
// A query (F frames x P fingerprints x a grid or per-frame windows) goes
// through three states:
//  queued   : descriptor copied at submit, waiting in FIFO order;
//  admitted : its device memory (frames if they came from the host,
//             residuals, work items, per-candidate results, output) fitted the
//             context's HBM budget; ingest (frame copy, noise residual, item
//             upload) runs on the copy stream and overlaps the compute stream;
//  done     : its last candidate has been scored and its per-(frame,
//             fingerprint) arg-max copied to the host.
// The compute stream runs waves of up to `wave` candidates.  A wave takes the
// next unlaunched candidates of the admitted queries of one frame size and
// storage type in admission order, so the tail of one query and the head of
// the next share launches: queries that arrive while others run join the next
// waves instead of waiting for an idle GPU.  Waves use per-slot indirection
// tables (item, result, residual frame), so the kernels are those of
// eis_grid_search and a query's results do not depend on what it was batched
// with.
//
// Two request loops run the waves (prnu_server_set_loop; device by default):
//  host   : the server thread forms each wave's tables and launches its
//           kernels;
//  device : for frame sizes with compile-time-planned kernels, one CUDA graph
//           per size class holds the whole loop.  A WHILE node repeats a body:
//           a scheduler kernel takes the next candidates of the ready queries
//           from a host-mapped ring, builds the wave tables on the device and
//           picks the branch of a SWITCH node that holds the wave kernels
//           in the smallest grids that fit the wave (shared forward units or
//           not; 16, 32, ... candidates and units).  A completion kernel
//           then writes the arg-max of every query the wave finished into
//           host-mapped memory and raises its done flag.  The host thread only admits queries
//           (memory, ingest, one ring entry each), relaunches a size class's
//           graph when it has drained or used its wave budget, and reports
//           queries whose done flag is up.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "search_fixed.h"
#include "server.h"
#include "wave_loop.h"

namespace prnu {

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxFrameSlots = 8192;
constexpr int kMaxFpSlots = 1024;
constexpr int kWaveSlots = 8;
constexpr int kMaxWave = 256;
// per wave: item pointers [kMaxWave], result pointers [kMaxWave], then the
// forward units' first slots [kMaxWave + 1] and each slot's unit [kMaxWave] (int)
constexpr size_t kWaveTabBytes = sizeof(void*) * 2 * kMaxWave + sizeof(int) * (2 * kMaxWave + 1);
constexpr size_t kMaxQueued = 4096;
constexpr int kArenaBlocks = 256;
constexpr size_t kArenaBlock = 64 * 1024;   // results of up to 2048 (frame, fingerprint) pairs

double ms_between(Clock::time_point t0, Clock::time_point t1) {
  return std::chrono::duration<double, std::milli>(t1 - t0).count();
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

__global__ void k_set_frame_ptrs(const void** __restrict__ dst, const char* __restrict__ base, int F,
                                 size_t frame_bytes) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < F) dst[f] = base + (size_t)f * frame_bytes;
}

__global__ void k_set_fpdesc(FpDesc* __restrict__ dst, FpDesc v) { *dst = v; }

// ---------------------------------------------------------------- device-resident loop

constexpr int kRing = 1024;       // queries of one size class admitted and not yet reported
constexpr int kLoopWaves = 32;    // waves per launch of a size class's loop

}  // namespace

struct Server::Impl {
  struct DevLoop;
  struct Query {
    uint64_t id = 0;
    int F = 0, H = 0, W = 0, P = 0, dtype = 0, flags = 0;
    size_t pitch = 0;
    prnu_grid grid{};
    const uint8_t* frames = nullptr;
    bool host_frames = false;
    std::vector<std::shared_ptr<Fingerprint>> fps;
    std::vector<prnu_window> windows;
    bool has_windows = false;
    Tuning tn;                     // launch configuration, read at submit
    size_t bytes = 0;
    char* dmem = nullptr;          // one pool allocation, carved below
    uint8_t* d_frames = nullptr;
    void* d_resid = nullptr;
    WorkItem* d_items = nullptr;
    CandResult* d_results = nullptr;
    int* d_groups = nullptr;
    prnu_result* d_out = nullptr;
    unsigned long long* d_acc = nullptr;
    double* d_partials = nullptr;
    int frame_slot0 = -1;
    std::vector<int> fp_slot;
    SearchCall call;               // host items and group table
    int next = 0;                  // items launched so far
    bool ingest_waited = false;
    cudaEvent_t ingest = nullptr;
    prnu_result* h_out = nullptr;  // pinned
    int arena_block = -1;
    std::vector<prnu_result> results;
    std::atomic<int> gpu_done{0};  // set by the stream callback (host loop) or on the done flag (device loop)
    DevLoop* loop = nullptr;       // device loop of its size class, or nullptr (host waves)
    long long ring_pos = -1;       // its position in that loop's ring
    bool reported = false;         // results copied out, resources released
    bool failed = false;
    int err = PRNU_OK;
    std::string errmsg;
    Clock::time_point t_submit, t_admit, t_done;
  };

  struct WaveSlot {
    void** h_tab = nullptr;        // pinned: item pointers, then result pointers
    void** d_tab = nullptr;
    cudaEvent_t ev = nullptr;
  };

  struct SizeKey {
    int H, W, dtype;
    bool operator<(const SizeKey& o) const {
      return H != o.H ? H < o.H : W != o.W ? W < o.W : dtype < o.dtype;
    }
  };

  prnu_ctx* ctx;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;       // wakes the server thread
  std::condition_variable done_cv;  // wakes pollers
  bool stopping = false;
  uint64_t next_id = 1;
  cudaStream_t s_comp = nullptr, s_copy = nullptr;
  cudaMemPool_t pool = nullptr;
  std::deque<std::shared_ptr<Query>> queued;
  std::vector<std::shared_ptr<Query>> admitted;
  std::map<uint64_t, std::shared_ptr<Query>> live;           // not yet retired by query_poll
  std::map<uint64_t, std::pair<double, double>> latency;     // id -> (queued ms, total ms)
  std::map<SizeKey, std::deque<std::shared_ptr<Query>>> active;
  std::vector<char> frame_used = std::vector<char>(kMaxFrameSlots, 0);
  const void** d_frame_ptrs = nullptr;
  float* d_scale = nullptr;
  FpDesc* d_fpdesc = nullptr;
  std::map<Fingerprint*, std::pair<int, int>> fp_slots;     // spectrum -> (slot, refs)
  std::vector<char> fp_used = std::vector<char>(kMaxFpSlots, 0);
  char* arena = nullptr;
  std::vector<char> arena_used = std::vector<char>(kArenaBlocks, 0);
  WaveSlot waves[kWaveSlots];
  int wave_next = 0;
  float2* ws_spec = nullptr;
  RowStat* ws_stats = nullptr;
  size_t ws_spec_bytes = 0, ws_stats_bytes = 0;
  prnu_server_stats st{};

  // The device-resident loop of one size class: its WaveLoop (graph,
  // scheduler state, wave tables) and the ring of admitted queries with their
  // ready and done flags (host-mapped).
  struct DevLoop {
    SizeKey key{};
    Tuning tn{};
    const FixedShape* fs = nullptr;
    int wave = 0;
    std::unique_ptr<WaveLoop> wl;
    DevRun* ring = nullptr;        // host pointer
    DevRun* d_ring = nullptr;      // its device pointer
    int* flags = nullptr;          // host pointer: tail, ready[kRing], done[kRing]
    int* d_flags = nullptr;
    long long appended = 0;
    std::deque<std::shared_ptr<Query>> runs;   // appended, not yet reported (ring order)
    bool dead = false;             // a launch failed: no further use
  };
  bool dev_mode = false;
  std::map<SizeKey, std::unique_ptr<DevLoop>> loops;   // nullptr: no planned kernels, host waves
  std::vector<std::unique_ptr<DevLoop>> retired;      // loops a device error retired
  cudaEvent_t loop_ev = nullptr;
  bool loop_running = false;
  DevLoop* loop_last = nullptr;    // the loop of the last launch
  int* h_loop_err = nullptr;       // pinned: the device flag after the last launch

  explicit Impl(prnu_ctx* c) : ctx(c) {
    PRNU_CUDA_TRY(cudaStreamCreateWithFlags(&s_comp, cudaStreamNonBlocking));
    PRNU_CUDA_TRY(cudaStreamCreateWithFlags(&s_copy, cudaStreamNonBlocking));
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = ctx->device;
    PRNU_CUDA_TRY(cudaMemPoolCreate(&pool, &props));
    unsigned long long keep = ~0ull;   // keep freed blocks for reuse by later queries
    PRNU_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    d_frame_ptrs = reinterpret_cast<const void**>(ctx_alloc(ctx, sizeof(void*) * kMaxFrameSlots));
    d_scale = reinterpret_cast<float*>(ctx_alloc(ctx, sizeof(float) * kMaxFrameSlots));
    d_fpdesc = reinterpret_cast<FpDesc*>(ctx_alloc(ctx, sizeof(FpDesc) * kMaxFpSlots));
    // mapped: the device loop's completion kernel writes query results here
    PRNU_CUDA_TRY(cudaHostAlloc((void**)&arena, kArenaBlock * kArenaBlocks, cudaHostAllocMapped));
    dev_mode = ctx->server_loop == PRNU_LOOP_DEVICE;
    if (dev_mode) {
      PRNU_CUDA_TRY(cudaEventCreateWithFlags(&loop_ev, cudaEventDisableTiming));
      PRNU_CUDA_TRY(cudaHostAlloc((void**)&h_loop_err, sizeof(int), cudaHostAllocDefault));
      *h_loop_err = 0;
    }
    for (auto& w : waves) {
      PRNU_CUDA_TRY(cudaHostAlloc((void**)&w.h_tab, kWaveTabBytes, cudaHostAllocDefault));
      w.d_tab = reinterpret_cast<void**>(ctx_alloc(ctx, kWaveTabBytes));
      PRNU_CUDA_TRY(cudaEventCreateWithFlags(&w.ev, cudaEventDisableTiming));
      PRNU_CUDA_TRY(cudaEventRecord(w.ev, s_comp));
    }
    th = std::thread([this] { loop(); });
  }

  ~Impl() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stopping = true;
    }
    cv.notify_all();
    if (th.joinable()) th.join();
    cudaStreamSynchronize(s_copy);
    cudaStreamSynchronize(s_comp);
    for (auto& q : admitted) release(*q);
    cudaStreamSynchronize(s_comp);
    for (auto& kv : loops) retired.push_back(std::move(kv.second));
    for (auto& L : retired) {
      if (!L) continue;
      L->wl.reset();
      if (L->ring) cudaFreeHost(L->ring);
      if (L->flags) cudaFreeHost(L->flags);
    }
    if (loop_ev) cudaEventDestroy(loop_ev);
    if (h_loop_err) cudaFreeHost(h_loop_err);
    for (auto& w : waves) {
      cudaFreeHost(w.h_tab);
      ctx_free(ctx, w.d_tab, kWaveTabBytes);
      cudaEventDestroy(w.ev);
    }
    ctx_free(ctx, d_frame_ptrs, sizeof(void*) * kMaxFrameSlots);
    ctx_free(ctx, d_scale, sizeof(float) * kMaxFrameSlots);
    ctx_free(ctx, d_fpdesc, sizeof(FpDesc) * kMaxFpSlots);
    if (ws_spec) ctx_free(ctx, ws_spec, ws_spec_bytes);
    if (ws_stats) ctx_free(ctx, ws_stats, ws_stats_bytes);
    cudaFreeHost(arena);
    cudaMemPoolDestroy(pool);
    cudaStreamDestroy(s_copy);
    cudaStreamDestroy(s_comp);
  }

  static size_t elem_size(int dtype) { return dtype == kF32 ? 4 : 2; }

  size_t query_bytes(const Query& q) const {
    const size_t px = (size_t)q.F * q.H * q.W;
    const size_t n = q.call.items.size();
    size_t b = 0;
    if (q.host_frames) b += align256(px);
    b += align256((size_t)q.F * padded_layout(q.H, q.W).fpitch * elem_size(q.dtype));   // zero-bordered residuals
    b += align256(sizeof(WorkItem) * n) + align256(sizeof(CandResult) * n);
    b += align256(sizeof(int) * ((size_t)q.F * q.P + 1)) + align256(sizeof(prnu_result) * (size_t)q.F * q.P);
    b += align256(sizeof(unsigned long long) * q.F) +
         align256(sizeof(double) * residual_partials_needed(q.F, q.H, q.W));
    return b;
  }

  // spectra: the wave's candidates, then, for a query whose fingerprints share
  // forward units, one slot per unit (at most one per candidate of the wave);
  // row statistics: the candidates
  size_t workspace_bytes(int H, int W, int wave, bool units) const {
    return (units ? 2 : 1) * (size_t)wave * H * (W / 2) * sizeof(float2) + (size_t)wave * H * sizeof(RowStat);
  }

  // ---------------------------------------------------------------- submit / poll (user threads)

  int submit(const prnu_query* pq, uint64_t* qid) {
    PRNU_CHECK_ARG(pq && qid, "NULL argument");
    PRNU_CHECK_ARG(pq->F >= 1 && pq->P >= 1, "a query needs F >= 1 frames and P >= 1 fingerprints");
    PRNU_CHECK_ARG(pq->frames && pq->fp_handles, "NULL frames or fingerprint handles");
    validate_shape(pq->H, pq->W);
    PRNU_CHECK_ARG(pq->dtype == kF32 || pq->dtype == kF16 || pq->dtype == kBF16, "unknown residual dtype");
    PRNU_CHECK_ARG((pq->flags & ~(PRNU_WEIGHT_BY_INTENSITY | PRNU_NORMALISE)) == 0, "unknown flags");
    PRNU_CHECK_ARG(pq->F <= kMaxFrameSlots / 2, "too many frames in one query");
    auto q = std::make_shared<Query>();
    q->F = pq->F;
    q->H = pq->H;
    q->W = pq->W;
    q->P = pq->P;
    q->dtype = pq->dtype;
    q->flags = pq->flags;
    q->pitch = pq->pitch ? pq->pitch : (size_t)pq->W;
    PRNU_CHECK_ARG(q->pitch >= (size_t)q->W, "pitch < W");
    q->grid = pq->grid;
    q->frames = pq->frames;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, pq->frames) != cudaSuccess) cudaGetLastError();
    q->host_frames = !(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    if (pq->windows) {
      q->windows.assign(pq->windows, pq->windows + pq->F);
      q->has_windows = true;
    }
    bool unit_major = false;
    {
      std::lock_guard<std::recursive_mutex> lk(ctx->mu);
      for (int p = 0; p < pq->P; ++p) {
        auto it = ctx->fps.find(pq->fp_handles[p]);
        if (it == ctx->fps.end())
          throw Error{PRNU_ENOTFOUND, "unknown fingerprint handle " + std::to_string(pq->fp_handles[p])};
        PRNU_CHECK_ARG(it->second->H == q->H && it->second->W == q->W, "fingerprint size differs from the frames");
        q->fps.push_back(it->second);
      }
      q->tn = tuning_for(ctx, q->H, q->W);
      // the fingerprints of one (frame, node) share its forward pass; a unit
      // (P items) never spans two waves
      unit_major = share_forward(ctx, q->H, q->W, q->P, false) && q->P <= kMaxWave;
    }
    build_items(q->grid, q->has_windows ? q->windows.data() : nullptr, q->F, q->P, q->call, unit_major);
    q->call.F = q->F;
    q->call.H = q->H;
    q->call.W = q->W;
    q->bytes = query_bytes(*q);
    const int wmax = dev_mode ? kLoopMaxWave : kMaxWave;   // the device loop's waves may be larger
    if (q->bytes + workspace_bytes(q->H, q->W, std::max(1, std::min(q->tn.wave, wmax)), unit_major) > ctx->budget)
      throw Error{PRNU_ENOMEM, "the query alone exceeds the HBM budget"};
    std::lock_guard<std::mutex> lk(mu);
    if (queued.size() >= kMaxQueued) throw Error{PRNU_EAGAIN, "query queue full"};
    q->id = next_id++;
    q->t_submit = Clock::now();
    queued.push_back(q);
    live[q->id] = q;
    *qid = q->id;
    cv.notify_all();
    return PRNU_OK;
  }

  int poll(uint64_t qid, prnu_result* out, int64_t timeout_us) {
    std::unique_lock<std::mutex> lk(mu);
    auto it = live.find(qid);
    if (it == live.end()) throw Error{PRNU_ENOTFOUND, "unknown or retired query id"};
    auto q = it->second;
    auto finished = [&] { return q->reported; };
    if (!finished()) {
      if (timeout_us == 0) return PRNU_EAGAIN;
      if (timeout_us < 0) done_cv.wait(lk, finished);
      else done_cv.wait_for(lk, std::chrono::microseconds(timeout_us), finished);
      if (!finished()) return PRNU_ETIMEOUT;
    }
    live.erase(qid);
    if (q->failed) throw Error{q->err ? q->err : PRNU_ECUDA, q->errmsg};
    if (out) memcpy(out, q->results.data(), sizeof(prnu_result) * q->results.size());
    return PRNU_OK;
  }

  // ---------------------------------------------------------------- server thread (holds mu)

  static void CUDART_CB on_done(void* p) {
    // CUDA callback thread: no CUDA calls here
    auto* q = static_cast<Query*>(p);
    q->t_done = Clock::now();
    q->gpu_done.store(1);
  }

  int alloc_frames(int F) {
    for (int s = 0; s + F <= kMaxFrameSlots;) {
      int k = 0;
      while (k < F && !frame_used[s + k]) ++k;
      if (k == F) {
        for (int i = 0; i < F; ++i) frame_used[s + i] = 1;
        return s;
      }
      s += k + 1;
    }
    return -1;
  }

  int take_fp_slot(const std::shared_ptr<Fingerprint>& f) {
    auto it = fp_slots.find(f.get());
    if (it != fp_slots.end()) {
      it->second.second++;
      return it->second.first;
    }
    for (int s = 0; s < kMaxFpSlots; ++s)
      if (!fp_used[s]) {
        fp_used[s] = 1;
        fp_slots[f.get()] = {s, 1};
        k_set_fpdesc<<<1, 1, 0, s_copy>>>(d_fpdesc + s, fp_desc(*f));
        PRNU_CUDA_TRY(cudaGetLastError());
        return s;
      }
    return -1;
  }

  void release(Query& q) {
    if (q.frame_slot0 >= 0)
      for (int i = 0; i < q.F; ++i) frame_used[q.frame_slot0 + i] = 0;
    q.frame_slot0 = -1;
    for (size_t p = 0; p < q.fp_slot.size(); ++p) {
      auto it = fp_slots.find(q.fps[p].get());
      if (it != fp_slots.end() && --it->second.second == 0) {
        fp_used[it->second.first] = 0;
        fp_slots.erase(it);
      }
    }
    q.fp_slot.clear();
    if (q.dmem) {
      cudaFreeAsync(q.dmem, s_comp);
      ctx->used -= q.bytes;
      st.admitted_bytes_now -= q.bytes;
      q.dmem = nullptr;
    }
    if (q.ingest) cudaEventDestroy(q.ingest);
    q.ingest = nullptr;
    if (q.arena_block >= 0) arena_used[q.arena_block] = 0;
    else if (q.h_out) cudaFreeHost(q.h_out);
    q.arena_block = -1;
    q.h_out = nullptr;
  }

  // spectrum slots and row-statistics slots (candidates) for frames of H x W
  void ensure_workspace(int H, int W, int spec_slots, int stat_slots) {
    const size_t sb = (size_t)spec_slots * H * (W / 2) * sizeof(float2);
    const size_t tb = (size_t)stat_slots * H * sizeof(RowStat);
    if (sb <= ws_spec_bytes && tb <= ws_stats_bytes) return;
    PRNU_CUDA_TRY(cudaStreamSynchronize(s_comp));
    if (ws_spec) ctx_free(ctx, ws_spec, ws_spec_bytes);
    if (ws_stats) ctx_free(ctx, ws_stats, ws_stats_bytes);
    ws_spec = nullptr;
    ws_stats = nullptr;   // device loops rebuild their graphs for the new pointers before their next launch
    ws_spec_bytes = std::max(sb, ws_spec_bytes);
    ws_stats_bytes = std::max(tb, ws_stats_bytes);
    ws_spec = reinterpret_cast<float2*>(ctx_alloc(ctx, ws_spec_bytes));
    ws_stats = reinterpret_cast<RowStat*>(ctx_alloc(ctx, ws_stats_bytes));
  }

  // Admit the head of the queue; false if it does not fit yet.
  bool admit(const std::shared_ptr<Query>& qp) {
    Query& q = *qp;
    DevLoop* L = dev_mode ? loop_for(q) : nullptr;   // nullptr: host waves
    if (L && (int)L->runs.size() >= kRing) return false;
    const int wave = L ? L->wave : std::max(1, std::min(q.tn.wave, kMaxWave));
    // spectra: the wave's candidates, then one slot per forward unit (a
    // device loop's branches are rebuilt for the slots there are)
    ensure_workspace(q.H, q.W, (q.call.share > 1 ? 2 : 1) * wave, wave);
    if (ctx->used.load() + q.bytes > ctx->budget) return false;
    const int slot0 = alloc_frames(q.F);
    if (slot0 < 0) return false;
    q.frame_slot0 = slot0;
    const size_t outb = sizeof(prnu_result) * (size_t)q.F * q.P;
    if (outb <= kArenaBlock) {
      for (int b = 0; b < kArenaBlocks; ++b)
        if (!arena_used[b]) {
          arena_used[b] = 1;
          q.arena_block = b;
          q.h_out = reinterpret_cast<prnu_result*>(arena + (size_t)b * kArenaBlock);
          break;
        }
      if (q.arena_block < 0) {
        release(q);
        return false;
      }
    } else {
      PRNU_CUDA_TRY(cudaHostAlloc((void**)&q.h_out, outb, cudaHostAllocMapped));
    }
    for (auto& f : q.fps) {
      const int s = take_fp_slot(f);
      if (s < 0) {
        release(q);
        throw Error{PRNU_ENOMEM, "fingerprint table full"};
      }
      q.fp_slot.push_back(s);
    }
    void* p = nullptr;
    if (cudaMallocFromPoolAsync(&p, q.bytes, pool, s_copy) != cudaSuccess) {
      cudaGetLastError();
      release(q);
      throw Error{PRNU_ENOMEM, "device allocation for the query failed"};
    }
    q.dmem = reinterpret_cast<char*>(p);
    ctx->used += q.bytes;
    st.admitted_bytes_now += q.bytes;
    st.admitted_bytes_peak = std::max(st.admitted_bytes_peak, st.admitted_bytes_now);
    const size_t px = (size_t)q.F * q.H * q.W;
    const size_t n = q.call.items.size();
    char* c = q.dmem;
    if (q.host_frames) {
      q.d_frames = reinterpret_cast<uint8_t*>(c);
      c += align256(px);
    }
    q.d_resid = c;
    const size_t resid_bytes = (size_t)q.F * padded_layout(q.H, q.W).fpitch * elem_size(q.dtype);
    c += align256(resid_bytes);
    q.d_items = reinterpret_cast<WorkItem*>(c);
    c += align256(sizeof(WorkItem) * n);
    q.d_results = reinterpret_cast<CandResult*>(c);
    c += align256(sizeof(CandResult) * n);
    q.d_groups = reinterpret_cast<int*>(c);
    c += align256(sizeof(int) * ((size_t)q.F * q.P + 1));
    q.d_out = reinterpret_cast<prnu_result*>(c);
    c += align256(outb);
    q.d_acc = reinterpret_cast<unsigned long long*>(c);
    c += align256(sizeof(unsigned long long) * q.F);
    q.d_partials = reinterpret_cast<double*>(c);
    for (auto& it : q.call.items) {   // global frame and fingerprint slots
      it.fp = q.fp_slot[it.fp];
      it.frame = q.frame_slot0 + it.frame;
    }
    for (auto& f : q.fps) PRNU_CUDA_TRY(cudaStreamWaitEvent(s_copy, f->ready, 0));
    const uint8_t* frames = q.frames;
    size_t pitch = q.pitch;
    if (q.host_frames) {
      PRNU_CUDA_TRY(cudaMemcpy2DAsync(q.d_frames, q.W, q.frames, q.pitch, q.W, (size_t)q.F * q.H,
                                      cudaMemcpyHostToDevice, s_copy));
      frames = q.d_frames;
      pitch = q.W;
    }
    // residuals go straight into the zero-bordered layout every search kernel here reads
    const ResidLayout lay = padded_layout(q.H, q.W);
    PRNU_CUDA_TRY(cudaMemsetAsync(q.d_resid, 0, resid_bytes, s_copy));
    launch_residual(frames, q.F, q.H, q.W, pitch, q.flags, q.dtype, q.d_resid, d_scale + q.frame_slot0, q.d_acc,
                    q.d_partials, (int)residual_partials_needed(q.F, q.H, q.W), s_copy, ctx->launches, &lay);
    k_set_frame_ptrs<<<(q.F + 127) / 128, 128, 0, s_copy>>>(d_frame_ptrs + q.frame_slot0,
                                                            reinterpret_cast<const char*>(q.d_resid), q.F,
                                                            lay.fpitch * elem_size(q.dtype));
    PRNU_CUDA_TRY(cudaGetLastError());
    PRNU_CUDA_TRY(cudaMemcpyAsync(q.d_items, q.call.items.data(), sizeof(WorkItem) * n, cudaMemcpyHostToDevice,
                                  s_copy));
    PRNU_CUDA_TRY(cudaMemcpyAsync(q.d_groups, q.call.group_start.data(), sizeof(int) * q.call.group_start.size(),
                                  cudaMemcpyHostToDevice, s_copy));
    PRNU_CUDA_TRY(cudaEventCreateWithFlags(&q.ingest, cudaEventDisableTiming));
    PRNU_CUDA_TRY(cudaEventRecord(q.ingest, s_copy));
    st.server_launches += 5;
    q.t_admit = Clock::now();
    admitted.push_back(qp);
    if (L) {
      append_run(*L, qp);
    } else {
      active[SizeKey{q.H, q.W, q.dtype}].push_back(qp);
    }
    return true;
  }

  // ---------------------------------------------------------------- device loop (holds mu)

  // The device loop of q's size class; nullptr where the size has no planned
  // kernels for q's tuning (its queries take host waves).
  DevLoop* loop_for(const Query& q) {
    const SizeKey key{q.H, q.W, q.dtype};
    auto it = loops.find(key);
    if (it != loops.end() && it->second && it->second->dead) {
      retired.push_back(std::move(it->second));   // kept until its queries are reported
      loops.erase(it);
      it = loops.end();
    }
    if (it != loops.end()) return it->second.get();
    const FixedShape* fs = q.tn.variant >= 0 ? find_fixed(q.H, q.W) : nullptr;
    if (!fs || !fixed_supports(*fs, q.H, q.tn.ppb)) {
      loops[key] = nullptr;
      return nullptr;
    }
    auto L = std::make_unique<DevLoop>();
    L->key = key;
    L->tn = q.tn;
    L->fs = fs;
    L->wave = std::max(1, std::min(q.tn.wave, kLoopMaxWave));   // the device tables hold up to 1024
    L->wl.reset(new WaveLoop(ctx));
    PRNU_CUDA_TRY(cudaHostAlloc((void**)&L->ring, sizeof(DevRun) * kRing, cudaHostAllocMapped));
    PRNU_CUDA_TRY(cudaHostAlloc((void**)&L->flags, sizeof(int) * (1 + 2 * kRing), cudaHostAllocMapped));
    memset(L->ring, 0, sizeof(DevRun) * kRing);
    memset(L->flags, 0, sizeof(int) * (1 + 2 * kRing));
    PRNU_CUDA_TRY(cudaHostGetDevicePointer((void**)&L->d_ring, L->ring, 0));
    PRNU_CUDA_TRY(cudaHostGetDevicePointer((void**)&L->d_flags, L->flags, 0));
    DevLoop* r = L.get();
    loops[key] = std::move(L);
    return r;
  }

  // Append an admitted query to its loop's ring: flags cleared, entry
  // written, ready raised on the copy stream after its ingest, then the tail
  // moved (the scheduler reads the tail, then the entry).
  void append_run(DevLoop& L, const std::shared_ptr<Query>& qp) {
    Query& q = *qp;
    const int slot = (int)(L.appended % kRing);
    volatile int* fl = L.flags;
    fl[1 + slot] = 0;
    fl[1 + kRing + slot] = 0;
    DevRun r{};
    r.items = q.d_items;
    r.results = q.d_results;
    r.groups = q.d_groups;
    PRNU_CUDA_TRY(cudaHostGetDevicePointer((void**)&r.out, q.h_out, 0));
    r.n = (int)q.call.items.size();
    r.share = std::max(q.call.share, 1);
    r.ngroups = q.F * q.P;
    L.ring[slot] = r;
    launch_mark_ready(L.d_flags + 1 + slot, s_copy);
    std::atomic_thread_fence(std::memory_order_seq_cst);
    q.loop = &L;
    q.ring_pos = L.appended;
    ++L.appended;
    fl[0] = (int)L.appended;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    L.runs.push_back(qp);
  }

  // What the size class's graph holds fixed: the shared tables, the current
  // workspace, the ring and its flags.
  WaveLoopConfig loop_config(const DevLoop& L) const {
    WaveLoopConfig c;
    c.fs = L.fs;
    c.variant = L.tn.variant;
    c.ppb = L.tn.ppb;
    c.col_log2 = L.tn.col_log2;
    c.H = L.key.H;
    c.W = L.key.W;
    c.rdtype = L.key.dtype;
    c.wave = L.wave;
    c.budget = kLoopWaves;
    c.fp_f32 = L.key.dtype == kF32 ? 1 : 0;   // half residuals: FP16 fingerprints expected (FP32 ones still correct)
    c.spec = ws_spec;
    c.stats = ws_stats;
    const size_t slot = (size_t)L.key.H * (L.key.W / 2) * sizeof(float2);
    c.spec_slots = (int)std::min<size_t>(ws_spec_bytes / slot, 1 << 20);
    c.frame_ptrs = d_frame_ptrs;
    c.fps = d_fpdesc;
    c.scale = d_scale;
    c.err = ctx->d_err;
    c.stall = ctx->debug_stall;
    c.ring = L.d_ring;
    c.tail = L.d_flags;
    c.ready = L.d_flags + 1;
    c.done = L.d_flags + 1 + kRing;
    c.ring_size = kRing;
    return c;
  }

  // One launch at a time on the compute stream: when the previous one has
  // ended, the size class whose oldest unfinished query (ingest complete) was
  // admitted first gets the next launch.
  void launch_loops() {
    if (loop_running) {
      if (cudaEventQuery(loop_ev) == cudaErrorNotReady) return;
      loop_running = false;
      if (*h_loop_err && loop_last) {
        // a bounded device-side wait gave up in that launch: its size class's
        // unreported queries fail, and the loop is not used again
        *h_loop_err = 0;
        PRNU_CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s_comp));
        loop_last->dead = true;
        const Error e{PRNU_EDEVICE_ABORT, "a bounded device-side wait timed out in the server's loop"};
        for (auto& qp : loop_last->runs)
          if (!qp->reported && !qp->gpu_done.load()) fail(*qp, e);
      }
    }
    DevLoop* best = nullptr;
    Clock::time_point oldest = Clock::time_point::max();
    for (auto& kv : loops) {
      DevLoop* L = kv.second.get();
      if (!L || L->dead) continue;
      for (auto& qp : L->runs) {
        if (qp->gpu_done.load() || qp->failed) continue;
        if (cudaEventQuery(qp->ingest) != cudaSuccess) break;
        if (qp->t_admit < oldest) {
          oldest = qp->t_admit;
          best = L;
        }
        break;
      }
    }
    if (!best) return;
    try {
      best->wl->ensure(loop_config(*best));
      best->wl->launch(s_comp);
      PRNU_CUDA_TRY(cudaMemcpyAsync(h_loop_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, s_comp));
      PRNU_CUDA_TRY(cudaEventRecord(loop_ev, s_comp));
      loop_last = best;
      loop_running = true;
      st.server_launches += 1;
    } catch (const Error& e) {
      best->dead = true;   // its ring may still name these queries: never launch it again
      for (auto& qp : best->runs)
        if (!qp->reported) fail(*qp, e);
    }
  }

  // The size class with the oldest unlaunched work, or active.end().
  std::map<SizeKey, std::deque<std::shared_ptr<Query>>>::iterator pick() {
    auto best = active.end();
    Clock::time_point oldest = Clock::time_point::max();
    for (auto it = active.begin(); it != active.end(); ++it) {
      while (!it->second.empty() &&
             (it->second.front()->failed || it->second.front()->next >= (int)it->second.front()->call.items.size()))
        it->second.pop_front();
      if (!it->second.empty() && it->second.front()->t_admit < oldest) {
        oldest = it->second.front()->t_admit;
        best = it;
      }
    }
    return best;
  }

  void launch_wave(std::map<SizeKey, std::deque<std::shared_ptr<Query>>>::iterator best, WaveSlot& slot) {
    const SizeKey key = best->first;
    const int H = key.H, W = key.W;
    const Tuning tn = best->second.front()->tn;
    // the twiddle offsets are fixed when the context is created
    const FftPlan prow = make_plan(W, ctx->tw_off), pcol = make_plan(H, ctx->tw_off);
    int rowT, rowMB;
    row_launch_shape(prow, &rowT, &rowMB);
    const int wave = std::max(1, std::min(tn.wave, kMaxWave));
    void** hi = slot.h_tab;
    void** hr = slot.h_tab + kMaxWave;
    int* hu = reinterpret_cast<int*>(slot.h_tab + 2 * kMaxWave);   // forward units' first slots
    int* hs = hu + kMaxWave + 1;                                      // unit of each slot
    int count = 0, nunits = 0;
    bool grouped = false, fp_f32 = false;
    std::vector<Query*> finished;
    for (auto& qp : best->second) {
      if (count >= wave) break;
      Query& q = *qp;
      const int n = (int)q.call.items.size();
      if (q.failed || q.next >= n) continue;
      // whole forward units only: a unit (the fingerprints of one frame and
      // node, share items) never spans two waves
      const int S = std::max(q.call.share, 1);
      const int take = std::min(wave - count, n - q.next) / S * S;
      if (take == 0) break;
      if (!q.ingest_waited) {
        PRNU_CUDA_TRY(cudaStreamWaitEvent(s_comp, q.ingest, 0));
        q.ingest_waited = true;
      }
      for (int k = 0; k < take; ++k) {
        hi[count + k] = q.d_items + q.next + k;
        hr[count + k] = q.d_results + q.next + k;
      }
      for (int u = 0; u < take / S; ++u) {
        for (int k = 0; k < S; ++k) hs[count + u * S + k] = nunits;
        hu[nunits++] = count + u * S;
      }
      grouped = grouped || S > 1;
      for (auto& f : q.fps) fp_f32 = fp_f32 || f->dtype == kF32;
      count += take;
      q.next += take;
      if (q.next == n) finished.push_back(&q);
    }
    hu[nunits] = count;
    // the candidates' slots, then (grouped wave) one per forward unit
    ensure_workspace(H, W, count + (grouped ? nunits : 0), count);
    PRNU_CUDA_TRY(cudaMemcpyAsync(slot.d_tab, slot.h_tab, kWaveTabBytes, cudaMemcpyHostToDevice, s_comp));
    PassArgs a{};
    a.err = ctx->d_err;
    a.rdtype = key.dtype;
    const ResidLayout lay = padded_layout(H, W);
    a.rpitch = lay.rpitch;
    a.fpitch = lay.fpitch;
    a.roff = lay.roff;
    a.H = H;
    a.W = W;
    a.nitems = count;
    a.spec = ws_spec;
    a.stats = ws_stats;
    a.fps = d_fpdesc;
    a.scale = d_scale;
    a.tw = ctx->d_tw;
    a.prow = prow;
    a.pcol = pcol;
    a.pairs_per_block = tn.ppb;
    a.col_log2 = tn.col_log2;
    a.row_threads = rowT;
    a.item_ptrs = reinterpret_cast<const WorkItem* const*>(slot.d_tab);
    a.result_ptrs = reinterpret_cast<CandResult* const*>(slot.d_tab + kMaxWave);
    a.frame_ptrs = d_frame_ptrs;
    // forward units of several items: the unit table; else one item per unit
    a.units = grouped ? reinterpret_cast<const int*>(slot.d_tab + 2 * kMaxWave) : nullptr;
    a.unit_of = grouped ? a.units + kMaxWave + 1 : nullptr;
    a.fp_f32 = fp_f32 ? 1 : 0;
    a.nunits = grouped ? nunits : count;
    a.share = 1;
    const FixedShape* fs = tn.variant >= 0 ? find_fixed(H, W) : nullptr;
    if (fs && !fixed_supports(*fs, H, tn.ppb)) fs = nullptr;
    if (fs) {
      launch_fixed_wave(a, *fs, tn.variant, s_comp, ctx->launches);
    } else {
      launch_row_forward(a, true, nullptr, nullptr, s_comp, ctx->launches);
      launch_col(a, 0, nullptr, nullptr, nullptr, s_comp, ctx->launches);
      launch_row_inverse(a, nullptr, s_comp, ctx->launches);
      launch_finalize(a, s_comp, ctx->launches);
    }
    PRNU_CUDA_TRY(cudaEventRecord(slot.ev, s_comp));
    st.server_launches += 4;
    st.candidates_done += count;
    for (Query* q : finished) {
      launch_argmax(q->d_results, q->d_items, q->d_groups, q->F * q->P, q->call.share, q->d_out, nullptr, q->H, q->W,
                    s_comp, ctx->launches);
      PRNU_CUDA_TRY(cudaMemcpyAsync(q->h_out, q->d_out, sizeof(prnu_result) * (size_t)q->F * q->P,
                                    cudaMemcpyDeviceToHost, s_comp));
      PRNU_CUDA_TRY(cudaLaunchHostFunc(s_comp, on_done, q));
      st.server_launches += 1;
    }
  }

  void fail(Query& q, const Error& e) {
    q.failed = true;
    q.err = e.code;
    q.errmsg = e.msg;
    q.t_done = Clock::now();
  }

  // results out, resources back, pollers woken
  bool report_finished() {
    bool any = false;
    for (size_t i = 0; i < admitted.size();) {
      Query& q = *admitted[i];
      if (q.loop && !q.failed && !q.gpu_done.load()) {
        const volatile int* fl = q.loop->flags;
        const int dv = fl[1 + kRing + (int)(q.ring_pos % kRing)];
        if (dv == 2) {
          fail(q, Error{PRNU_EDEVICE_ABORT, "a bounded device-side wait timed out in the server's loop"});
        } else if (dv) {
          std::atomic_thread_fence(std::memory_order_acquire);
          q.t_done = Clock::now();
          q.gpu_done.store(1);
          st.candidates_done += q.call.items.size();
        }
      }
      if (q.gpu_done.load() || q.failed) {
        if (!q.failed) {
          q.results.assign(q.h_out, q.h_out + (size_t)q.F * q.P);
          latency[q.id] = {ms_between(q.t_submit, q.t_admit), ms_between(q.t_submit, q.t_done)};
          st.queries_done++;
        }
        release(q);
        q.reported = true;
        admitted[i] = admitted.back();
        admitted.pop_back();
        any = true;
      } else {
        ++i;
      }
    }
    while (latency.size() > 100000) latency.erase(latency.begin());
    for (auto& kv : loops)
      if (kv.second)
        while (!kv.second->runs.empty() && kv.second->runs.front()->reported) kv.second->runs.pop_front();
    return any;
  }

  void loop() {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stopping) {
      bool progressed = report_finished();
      while (!queued.empty()) {
        auto q = queued.front();
        bool ok = false;
        try {
          ok = admit(q);
        } catch (const Error& e) {
          fail(*q, e);
          q->reported = true;
          queued.pop_front();
          progressed = true;
          continue;
        }
        if (!ok) break;
        queued.pop_front();
        progressed = true;
      }
      if (progressed) done_cv.notify_all();
      if (dev_mode) launch_loops();
      auto best = pick();
      if (best != active.end()) {
        WaveSlot& slot = waves[wave_next];
        wave_next = (wave_next + 1) % kWaveSlots;
        lk.unlock();
        cudaEventSynchronize(slot.ev);   // the slot's tables are free again
        lk.lock();
        try {
          auto again = pick();
          if (again != active.end()) launch_wave(again, slot);
        } catch (const Error& e) {
          for (auto& kv : active)
            for (auto& q : kv.second) fail(*q, e);
          active.clear();
        }
        continue;
      }
      if (!progressed) cv.wait_for(lk, std::chrono::microseconds(200));
    }
  }
};

Server::Server(prnu_ctx* ctx) : impl_(new Impl(ctx)) {}
Server::~Server() = default;
int Server::submit(const prnu_query* q, uint64_t* qid) { return impl_->submit(q, qid); }
int Server::poll(uint64_t qid, prnu_result* out, int64_t timeout_us) { return impl_->poll(qid, out, timeout_us); }
void Server::stats(prnu_server_stats* out) {
  std::lock_guard<std::mutex> lk(impl_->mu);
  *out = impl_->st;
}
bool Server::latency(uint64_t qid, double* queued_ms, double* total_ms) {
  std::lock_guard<std::mutex> lk(impl_->mu);
  auto it = impl_->latency.find(qid);
  if (it == impl_->latency.end()) return false;
  if (queued_ms) *queued_ms = it->second.first;
  if (total_ms) *total_ms = it->second.second;
  return true;
}

}  // namespace prnu

using namespace prnu;

namespace {

Server& server_of(prnu_ctx* ctx) {
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (!ctx->server) {
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    ctx->server.reset(new Server(ctx));
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  }
  return *ctx->server;
}

template <class Fn>
int serve_guard(Fn&& fn) {
  try {
    int rc = fn();
    if (rc == PRNU_OK) set_error("");
    return rc;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.code;
  } catch (const std::exception& e) {
    set_error(e.what());
    return PRNU_EINVAL;
  }
}

}  // namespace

extern "C" {

int query_submit(prnu_ctx* ctx, const prnu_query* q, uint64_t* qid) {
  return serve_guard([&] {
    PRNU_CHECK_ARG(ctx, "NULL context");
    return server_of(ctx).submit(q, qid);
  });
}

int query_poll(prnu_ctx* ctx, uint64_t qid, prnu_result* out, int64_t timeout_us) {
  return serve_guard([&] {
    PRNU_CHECK_ARG(ctx, "NULL context");
    return server_of(ctx).poll(qid, out, timeout_us);
  });
}

int query_latency(prnu_ctx* ctx, uint64_t qid, double* queued_ms, double* total_ms) {
  return serve_guard([&] {
    PRNU_CHECK_ARG(ctx, "NULL context");
    if (!server_of(ctx).latency(qid, queued_ms, total_ms))
      throw Error{PRNU_ENOTFOUND, "no finished query with this id"};
    return (int)PRNU_OK;
  });
}

int prnu_server_set_loop(prnu_ctx* ctx, int mode) {
  if (!ctx) {
    set_error("NULL context");
    return PRNU_EINVAL;
  }
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (mode != PRNU_LOOP_HOST && mode != PRNU_LOOP_DEVICE) {
    set_error("unknown server loop mode");
    return PRNU_EINVAL;
  }
  if (ctx->server && mode != ctx->server_loop) {
    set_error("the server has started: set its loop before the first query_submit");
    return PRNU_EINVAL;
  }
  ctx->server_loop = mode;
  set_error("");
  return PRNU_OK;
}

int prnu_server_stats_get(prnu_ctx* ctx, prnu_server_stats* out) {
  return serve_guard([&] {
    PRNU_CHECK_ARG(ctx && out, "NULL argument");
    server_of(ctx).stats(out);
    return (int)PRNU_OK;
  });
}

}  // extern "C"
