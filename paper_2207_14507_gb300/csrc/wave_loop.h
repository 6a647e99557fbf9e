// wave_loop.h -- the device-resident wave loop: one CUDA graph whose WHILE
// node repeats
//  - a scheduler kernel: the next candidates of the ready runs of a ring, in
//    whole forward units, into the wave's item, result and unit tables;
//  - a SWITCH node over wave shapes: the wave kernels of the compile-time
//    planned path, with grids for 16, 32, ... candidates (and forward units),
//    the smallest branch that holds the wave;
//  - a completion kernel: the arg-max of every run the wave finished, into
//    the run's result buffer, then the run's done flag.
// The query server runs one per frame size over a host-mapped ring of
// queries; eis_grid_search (prnu_tuning.persistent = 2) runs one over a
// single run, the call's work list.
#pragma once
#include "internal.h"
#include "search_fixed.h"

namespace prnu {

constexpr int kLoopMaxWave = 1024;  // wave table capacity

// One run of candidates: a query of the server, or one call's work list.
struct DevRun {
  const WorkItem* items;    // device [n]
  CandResult* results;      // device [n]
  const int* groups;        // device group table (SearchCall::group_start)
  prnu_result* out;         // [ngroups], device or host-mapped: the arg-max per group
  int n;                    // candidates
  int share;                // fingerprints per forward unit (1: none)
  int ngroups;              // groups the completion kernel reduces (0: none)
  int pad;
};

// Device state of one loop.
struct DevSched {
  int head;                 // ring position of the first run not fully scheduled
  int next;                 // its next candidate
  int waves;                // waves run by the current launch
  int counts[2];            // the current wave's items and forward units (PassArgs::d_counts)
  int ncomplete;            // runs whose last candidates are in the current wave
  int complete[kLoopMaxWave];
};

// What a loop's graph holds fixed; a different configuration rebuilds it.
struct WaveLoopConfig {
  const FixedShape* fs = nullptr;
  int variant = 0, ppb = 0, col_log2 = 0;   // the tuning of the planned kernels
  int H = 0, W = 0;
  int rdtype = 0;              // residual layout the wave kernels read
  int wave = 0;                // candidates per wave (<= kLoopMaxWave)
  int budget = 0;              // waves per launch (0: until no run is ready)
  int fp_f32 = 0;              // some fingerprint is FP32 (column-variant choice)
  float2* spec = nullptr;      // workspace spectra
  RowStat* stats = nullptr;
  int spec_slots = 0;          // spectra the workspace holds
  const void* resid = nullptr;              // residuals: frame_ptrs[f] if set, else resid + f * frame pitch
  const void* const* frame_ptrs = nullptr;
  const FpDesc* fps = nullptr;
  const float* scale = nullptr;
  int* err = nullptr;
  int stall = 0;
  const DevRun* ring = nullptr;             // ring_size runs, device-accessible
  const int* tail = nullptr;                // runs appended so far
  const int* ready = nullptr;               // [ring_size] ingest complete
  int* done = nullptr;                      // [ring_size] completion flags (2: an error was raised)
  int ring_size = 1;
  bool same(const WaveLoopConfig& o) const;
};

class WaveLoop {
 public:
  explicit WaveLoop(prnu_ctx* ctx);
  ~WaveLoop();
  WaveLoop(const WaveLoop&) = delete;
  WaveLoop& operator=(const WaveLoop&) = delete;
  // (re)capture the graph if c differs from the configuration it was built for
  void ensure(const WaveLoopConfig& c);
  // one launch on s: waves until no run is ready or the budget is used
  void launch(cudaStream_t s);
  // the scheduler back to the start of the ring (a ring of one run, reused)
  void rewind(cudaStream_t s);

 private:
  prnu_ctx* ctx_;
  char* dmem_ = nullptr;
  size_t dbytes_ = 0;
  DevSched* st_ = nullptr;
  const WorkItem** items_ = nullptr;
  CandResult** results_ = nullptr;
  int* units_ = nullptr;
  int* unit_of_ = nullptr;
  cudaStream_t cap_ = nullptr;
  cudaEvent_t ev_ = nullptr;       // recorded after each launch: the graph is not destroyed before it
  cudaGraph_t graph_ = nullptr;
  cudaGraphExec_t exec_ = nullptr;
  WaveLoopConfig cfg_{};
  bool built_ = false;
  void build();
  void capture(cudaGraph_t into, bool units, int items, int nunits);
};

// eis_grid_search's loop (prnu_tuning.persistent = 2): a WaveLoop over a ring
// of one run, the call's work list, in device memory, with no wave budget.
class BatchLoop {
 public:
  explicit BatchLoop(prnu_ctx* ctx);
  ~BatchLoop();
  BatchLoop(const BatchLoop&) = delete;
  BatchLoop& operator=(const BatchLoop&) = delete;
  // every wave of run r on s, in one graph launch (c: all but the ring fields)
  void run(WaveLoopConfig c, const DevRun& r, cudaStream_t s);
  // the same for the run a kernel earlier on s wrote into ring_entry()
  void run_written(WaveLoopConfig c, cudaStream_t s);
  DevRun* ring_entry() const { return reinterpret_cast<DevRun*>(mem_); }

 private:
  prnu_ctx* ctx_;
  WaveLoop wl_;
  char* mem_ = nullptr;    // the run, then tail, ready, done
  size_t bytes_ = 0;
};

// raise a ready flag (device-accessible memory) once the work before it on s is done
void launch_mark_ready(int* ready, cudaStream_t s);

}  // namespace prnu
