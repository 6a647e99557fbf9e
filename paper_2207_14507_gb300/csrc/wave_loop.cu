// wave_loop.cu -- the device-resident wave loop (wave_loop.h).
#include <algorithm>
#include <cstring>

#include "search_common.cuh"
#include "wave_loop.h"

namespace prnu {

namespace {

// The wave shapes a loop body holds, one branch each of its SWITCH node:
// shared forward units or not, and the grids' sizes (items, and forward
// units), so that a wave runs in the smallest branch that fits it.
constexpr int kMaxCases = 40;
struct CaseTable {
  int n;
  int grouped[kMaxCases];
  int items[kMaxCases];
  int units[kMaxCases];
};

__device__ __forceinline__ int ld_acquire_sys(const int* p) {
  int v;
  asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(int* p, int v) {
  asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__global__ void k_loop_begin(DevSched* st) { st->waves = 0; }

__global__ void k_set_run(DevRun* dst, DevRun v) { *dst = v; }

__global__ void k_loop_rewind(DevSched* st) {
  st->head = 0;
  st->next = 0;
}

// the work before it on its stream is done: raise the flag
__global__ void k_mark_ready(int* ready) {
  __threadfence_system();
  st_release_sys(ready, 1);
}

// the first branch of the case table that holds a wave, or ct.n
__device__ __forceinline__ int fit_case(const CaseTable& ct, int count, int nunits, bool grouped) {
  for (int k = 0; k < ct.n; ++k)
    if (ct.grouped[k] == (grouped ? 1 : 0) && ct.items[k] >= count && (!grouped || ct.units[k] >= nunits)) return k;
  return ct.n;
}

// One wave: up to `wave` candidates of the ready runs in ring order, whole
// forward units only (as many as a branch of the body holds), into the wave
// tables; the smallest branch that holds it; the loop goes on while it found
// candidates and the launch's wave budget (0: none) lasts.  One warp: lane 0
// plans the wave as segments (a run's next candidates), all lanes write the
// tables.
struct Segment {
  const WorkItem* items;
  CandResult* results;
  int count0, nunits0, take, S;
};

__global__ void __launch_bounds__(32) k_sched(DevSched* st, const DevRun* ring, int ring_size, const int* tail_p,
                                              const int* ready, int wave, int budget, const WorkItem** item_ptrs,
                                              CandResult** result_ptrs, int* units, int* unit_of,
                                              cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_case,
                                              CaseTable ct) {
  __shared__ Segment seg[kLoopMaxWave];
  __shared__ int s_nseg;
  const int lane = threadIdx.x;
  if (lane == 0) {
    const int tail = ld_acquire_sys(tail_p);
    int head = st->head, next = st->next, count = 0, nunits = 0, ncomp = 0, nseg = 0;
    bool grouped = false;
    while (count < wave && ncomp < kLoopMaxWave && head != tail) {
      const int slot = head % ring_size;
      if (ld_acquire_sys(ready + slot) == 0) break;   // ingest still running: keep arrival order
      const DevRun r = ring[slot];
      if (r.n <= 0) {                                  // nothing to score: complete at once
        st->complete[ncomp++] = head;
        ++head;
        next = 0;
        continue;
      }
      const int S = max(r.share, 1);
      int take = min(wave - count, r.n - next) / S * S;
      while (take > 0 && fit_case(ct, count + take, nunits + take / S, grouped || S > 1) == ct.n) take -= S;
      if (take == 0) break;
      seg[nseg++] = Segment{r.items + next, r.results + next, count, nunits, take, S};
      grouped = grouped || S > 1;
      count += take;
      nunits += take / S;
      next += take;
      if (next == r.n) {
        st->complete[ncomp++] = head;
        ++head;
        next = 0;
      }
    }
    units[nunits] = count;
    st->head = head;
    st->next = next;
    st->counts[0] = count;
    st->counts[1] = grouped ? nunits : count;
    st->ncomplete = ncomp;
    const int waves = st->waves + 1;
    st->waves = waves;
    s_nseg = nseg;
    const int c = count > 0 ? fit_case(ct, count, nunits, grouped) : ct.n;   // ct.n: no branch runs
    cudaGraphSetConditional(h_case, (unsigned)c);
    cudaGraphSetConditional(h_loop, count > 0 && (budget == 0 || waves < budget) ? 1u : 0u);
  }
  __syncwarp();
  const int nseg = s_nseg;
  for (int q = 0; q < nseg; ++q) {
    const Segment g = seg[q];
    for (int k = lane; k < g.take; k += 32) {
      item_ptrs[g.count0 + k] = g.items + k;
      result_ptrs[g.count0 + k] = g.results + k;
      unit_of[g.count0 + k] = g.nunits0 + k / g.S;
    }
    for (int u = lane; u < g.take / g.S; u += 32) units[g.nunits0 + u] = g.count0 + u * g.S;
  }
  __threadfence();
}

// The arg-max of every run the wave finished, into its result buffer, then
// its done flag: 1, or 2 if a bounded device-side wait has given up (the
// context's error flag err is raised: the results are not to be trusted).
// Block b takes finished runs b, b + gridDim.x, ...
__global__ void k_complete(const DevSched* st, const DevRun* ring, int ring_size, int* done, const int* err, int H,
                           int W) {
  const int ncomp = st->ncomplete;
  for (int c = blockIdx.x; c < ncomp; c += gridDim.x) {
    const int slot = st->complete[c] % ring_size;
    const DevRun r = ring[slot];
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int g = threadIdx.x >> 5; g < r.ngroups; g += nw)
      argmax_group(r.results, r.items, r.groups, max(r.share, 1), r.out, H, W, g, lane);
    __syncthreads();
    if (threadIdx.x == 0) {
      const int bad = err != nullptr && ld_acquire_sys(err) != 0;
      __threadfence_system();
      st_release_sys(done + slot, bad ? 2 : 1);
    }
    __syncthreads();
  }
}

// Plain and shared-forward waves with grids of 16, 32, ... up to `wave`
// items (and, shared, as many or fewer units), within `slots` workspace
// spectra (a shared wave takes items + units).
CaseTable case_table(int wave, int slots) {
  std::vector<int> caps;
  for (int c = 16; c < wave; c *= 2) caps.push_back(c);
  caps.push_back(wave);
  CaseTable ct{};
  auto add = [&](int g, int it, int un) {
    if (ct.n >= kMaxCases) return;
    ct.grouped[ct.n] = g;
    ct.items[ct.n] = it;
    ct.units[ct.n] = un;
    ++ct.n;
  };
  for (int it : caps)
    if (it <= slots) add(0, it, it);
  for (int it : caps)
    for (int un : caps)
      if (un <= it && it + un <= slots) add(1, it, un);
  return ct;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

bool WaveLoopConfig::same(const WaveLoopConfig& o) const {
  return fs == o.fs && variant == o.variant && ppb == o.ppb && col_log2 == o.col_log2 && H == o.H && W == o.W &&
         rdtype == o.rdtype && wave == o.wave && budget == o.budget && fp_f32 == o.fp_f32 && spec == o.spec &&
         stats == o.stats && spec_slots == o.spec_slots && resid == o.resid && frame_ptrs == o.frame_ptrs &&
         fps == o.fps && scale == o.scale && err == o.err && stall == o.stall && ring == o.ring && tail == o.tail &&
         ready == o.ready && done == o.done && ring_size == o.ring_size;
}

WaveLoop::WaveLoop(prnu_ctx* ctx) : ctx_(ctx) {
  const size_t o_items = align256(sizeof(DevSched));
  const size_t o_results = o_items + align256(sizeof(void*) * kLoopMaxWave);
  const size_t o_units = o_results + align256(sizeof(void*) * kLoopMaxWave);
  const size_t o_unit_of = o_units + align256(sizeof(int) * (kLoopMaxWave + 1));
  dbytes_ = o_unit_of + align256(sizeof(int) * kLoopMaxWave);
  dmem_ = reinterpret_cast<char*>(ctx_alloc(ctx_, dbytes_));
  PRNU_CUDA_TRY(cudaMemset(dmem_, 0, dbytes_));
  st_ = reinterpret_cast<DevSched*>(dmem_);
  items_ = reinterpret_cast<const WorkItem**>(dmem_ + o_items);
  results_ = reinterpret_cast<CandResult**>(dmem_ + o_results);
  units_ = reinterpret_cast<int*>(dmem_ + o_units);
  unit_of_ = reinterpret_cast<int*>(dmem_ + o_unit_of);
  PRNU_CUDA_TRY(cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking));
  PRNU_CUDA_TRY(cudaEventCreateWithFlags(&ev_, cudaEventDisableTiming));
}

WaveLoop::~WaveLoop() {
  if (ev_) {
    cudaEventSynchronize(ev_);
    cudaEventDestroy(ev_);
  }
  if (exec_) cudaGraphExecDestroy(exec_);
  if (graph_) cudaGraphDestroy(graph_);
  if (cap_) cudaStreamDestroy(cap_);
  if (dmem_) ctx_free(ctx_, dmem_, dbytes_);
}

void WaveLoop::ensure(const WaveLoopConfig& c) {
  if (built_ && cfg_.same(c)) return;
  cfg_ = c;
  build();
}

void WaveLoop::launch(cudaStream_t s) {
  PRNU_CUDA_TRY(cudaGraphLaunch(exec_, s));
  PRNU_CUDA_TRY(cudaEventRecord(ev_, s));
  ctx_->launches.n++;
}

void WaveLoop::rewind(cudaStream_t s) {
  k_loop_rewind<<<1, 1, 0, s>>>(st_);
  PRNU_CUDA_TRY(cudaGetLastError());
}

// The wave kernels of one branch, captured into `into`: grids for `items`
// candidates and `nunits` forward units (the unit slots follow the items'),
// the live counts read on the device.
void WaveLoop::capture(cudaGraph_t into, bool units, int items, int nunits) {
  const WaveLoopConfig& c = cfg_;
  const FftPlan prow = make_plan(c.W, ctx_->tw_off), pcol = make_plan(c.H, ctx_->tw_off);
  int rowT, rowMB;
  row_launch_shape(prow, &rowT, &rowMB);
  PassArgs a{};
  a.err = c.err;
  a.stall = c.stall;
  a.resid = c.resid;
  a.rdtype = c.rdtype;
  const ResidLayout lay = padded_layout(c.H, c.W);
  a.rpitch = lay.rpitch;
  a.fpitch = lay.fpitch;
  a.roff = lay.roff;
  a.H = c.H;
  a.W = c.W;
  a.nitems = items;
  a.spec = c.spec;
  a.stats = c.stats;
  a.fps = c.fps;
  a.scale = c.scale;
  a.tw = ctx_->d_tw;
  a.prow = prow;
  a.pcol = pcol;
  a.pairs_per_block = c.ppb;
  a.col_log2 = c.col_log2;
  a.row_threads = rowT;
  a.item_ptrs = items_;
  a.result_ptrs = results_;
  a.frame_ptrs = c.frame_ptrs;
  a.units = units ? units_ : nullptr;
  a.unit_of = units ? unit_of_ : nullptr;
  a.nunits = nunits;
  a.share = 1;
  a.fp_f32 = c.fp_f32;
  a.d_counts = st_->counts;
  LaunchCounter lc;
  PRNU_CUDA_TRY(cudaStreamBeginCaptureToGraph(cap_, into, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  try {
    launch_fixed_wave(a, *c.fs, c.variant, cap_, lc);
  } catch (...) {
    cudaGraph_t g;
    cudaStreamEndCapture(cap_, &g);
    cudaGetLastError();
    throw;
  }
  cudaGraph_t g;
  PRNU_CUDA_TRY(cudaStreamEndCapture(cap_, &g));
}

// loop begin -> WHILE { scheduler -> SWITCH { wave branches } -> completion }
void WaveLoop::build() {
  if (exec_) PRNU_CUDA_TRY(cudaEventSynchronize(ev_));   // the last launch of the old graph has ended
  if (exec_) cudaGraphExecDestroy(exec_);
  if (graph_) cudaGraphDestroy(graph_);
  exec_ = nullptr;
  graph_ = nullptr;
  built_ = false;
  const WaveLoopConfig& c = cfg_;
  PRNU_CHECK_ARG(c.fs && c.wave >= 1 && c.wave <= kLoopMaxWave && c.ring_size >= 1, "bad wave loop configuration");
  CaseTable ct = case_table(c.wave, c.spec_slots);
  if (ct.n == 0) throw Error{PRNU_ENOMEM, "no workspace for a wave of this frame size"};
  cudaGraph_t g;
  PRNU_CUDA_TRY(cudaGraphCreate(&g, 0));
  graph_ = g;
  cudaGraphConditionalHandle h_loop, h_case;
  PRNU_CUDA_TRY(cudaGraphConditionalHandleCreate(&h_loop, g, 1, cudaGraphCondAssignDefault));
  PRNU_CUDA_TRY(cudaGraphConditionalHandleCreate(&h_case, g, 0, cudaGraphCondAssignDefault));
  auto kernel_node = [](cudaGraphNode_t* n, cudaGraph_t gr, const cudaGraphNode_t* dep, void* fn, int grid,
                        int block, void** args) {
    cudaKernelNodeParams kp{};
    kp.func = fn;
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(block);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    PRNU_CUDA_TRY(cudaGraphAddKernelNode(n, gr, dep, dep ? 1 : 0, &kp));
  };
  cudaGraphNode_t n_begin, n_loop, n_sched, n_switch, n_done;
  DevSched* d_st = st_;
  void* bargs[] = {&d_st};
  kernel_node(&n_begin, g, nullptr, (void*)k_loop_begin, 1, 1, bargs);
  cudaGraphNodeParams wp{};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = h_loop;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  PRNU_CUDA_TRY(cudaGraphAddNode(&n_loop, g, &n_begin, nullptr, 1, &wp));
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  const DevRun* ring = c.ring;
  int ring_size = c.ring_size, wave = c.wave, budget = c.budget, H = c.H, W = c.W;
  const int* tail = c.tail;
  const int* ready = c.ready;
  int* done = c.done;
  const WorkItem** items = items_;
  CandResult** results = results_;
  int* units = units_;
  int* unit_of = unit_of_;
  void* sargs[] = {&d_st, &ring, &ring_size, &tail, &ready, &wave, &budget, &items, &results, &units,
                   &unit_of, &h_loop, &h_case, &ct};
  kernel_node(&n_sched, body, nullptr, (void*)k_sched, 1, 32, sargs);
  cudaGraphNodeParams sp{};
  sp.type = cudaGraphNodeTypeConditional;
  sp.conditional.handle = h_case;
  sp.conditional.type = cudaGraphCondTypeSwitch;
  sp.conditional.size = (unsigned)ct.n;
  PRNU_CUDA_TRY(cudaGraphAddNode(&n_switch, body, &n_sched, nullptr, 1, &sp));
  for (int k = 0; k < ct.n; ++k) capture(sp.conditional.phGraph_out[k], ct.grouped[k] != 0, ct.items[k], ct.units[k]);
  const DevSched* d_stc = d_st;
  const int* err = c.err;
  void* cargs[] = {&d_stc, &ring, &ring_size, &done, &err, &H, &W};
  kernel_node(&n_done, body, &n_switch, (void*)k_complete, 64, 256, cargs);
  PRNU_CUDA_TRY(cudaGraphInstantiate(&exec_, g, 0));
  built_ = true;
}

BatchLoop::BatchLoop(prnu_ctx* ctx) : ctx_(ctx), wl_(ctx) {
  bytes_ = 256 + 3 * sizeof(int);
  mem_ = reinterpret_cast<char*>(ctx_alloc(ctx_, bytes_));
  const int flags[3] = {1, 1, 0};   // one run appended, ready; not done
  PRNU_CUDA_TRY(cudaMemset(mem_, 0, bytes_));
  PRNU_CUDA_TRY(cudaMemcpy(mem_ + 256, flags, sizeof(flags), cudaMemcpyHostToDevice));
}

BatchLoop::~BatchLoop() {
  if (mem_) ctx_free(ctx_, mem_, bytes_);
}

void BatchLoop::run(WaveLoopConfig c, const DevRun& r, cudaStream_t s) {
  k_set_run<<<1, 1, 0, s>>>(ring_entry(), r);
  PRNU_CUDA_TRY(cudaGetLastError());
  run_written(c, s);
}

void BatchLoop::run_written(WaveLoopConfig c, cudaStream_t s) {
  int* flags = reinterpret_cast<int*>(mem_ + 256);
  c.ring = reinterpret_cast<const DevRun*>(mem_);
  c.tail = flags;
  c.ready = flags + 1;
  c.done = flags + 2;
  c.ring_size = 1;
  c.budget = 0;
  wl_.ensure(c);
  wl_.rewind(s);
  wl_.launch(s);
}

void launch_mark_ready(int* ready, cudaStream_t s) {
  k_mark_ready<<<1, 1, 0, s>>>(ready);
  PRNU_CUDA_TRY(cudaGetLastError());
}

}  // namespace prnu
