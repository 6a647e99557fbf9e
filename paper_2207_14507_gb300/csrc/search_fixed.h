// search_fixed.h -- registry of the compile-time-planned kernels (search_fixed.cu).
#pragma once
#include <vector>

#include "internal.h"

namespace prnu {

// one instantiated column-pass variant: columns per block, threads, shared
// memory; with tma the kernel moves its strip by TMA tile copies of br rows
// and takes a CUtensorMap of the workspace spectra as a second argument,
// otherwise each thread loads and stores its own elements
struct FixedCol {
  int nc;
  int threads;
  size_t smem;
  void* fn;
  bool tma;
  int br;
  int mode;   // 0 plain loads, 1 strip by TMA, 2 fingerprint by TMA into the strip buffer, 3/4 into its own region
};

// one instantiated pair of row kernels: row pairs per block, threads per pair
struct FixedRow {
  int ppb;
  int threads;               // per row pair, forward kernel
  int threads_inv;           // per row pair, inverse kernel
  size_t smem;
  void* fwd[kNumStoreLayouts];   // by residual storage type (kF32, kF16, kBF16, kF16P, kBF16P)
  void* inv;
  void* fin;                 // per-candidate PCE (one block per candidate)
  int fin_threads;
  size_t fin_smem;
};

// the persistent kernel of a shape: row pairs per task, columns per task,
// block size, shared memory, resident blocks per SM, by residual type
struct FixedPersist {
  int ppb, nc, threads;
  size_t smem;
  void* fn[3];
  int blocks_per_sm[3];
};

// Device state of one persistent launch: the ticket, the error flag, and the
// per-candidate completion counts of the four phases ([G] each), all zeroed
// before the launch.  S = workspace slots (spectra, row statistics).
struct PersistArgs {
  int* ticket;
  int* error;
  int* rf_done;
  int* col_done;
  int* ri_done;
  int* fin_done;
  int G;
  int S;
};

struct FixedShape {
  int W, H;
  std::vector<FixedRow> rows;
  std::vector<FixedCol> cols;
  FixedCol col_fwd, col_inv; // the column pass split for forward units (k_col_fwd_fx, k_col_inv_fx)
  FixedCol col_inv_sep;      // k_col_inv_fx with the fingerprint strip in its own region (mode 3/4), taken
                             // with a column variant of that mode; fn null where none is instantiated
  FixedCol col_inv_h;        // the same with a region for FP16 bins (mode 4) and more blocks per SM, taken
                             // instead when every fingerprint of the wave is FP16; fn null where none
  FixedPersist persist;
  // the row kernels with `ppb` pairs per block, else the first variant
  const FixedRow& row_for(int ppb) const {
    for (auto& r : rows)
      if (r.ppb == ppb) return r;
    return rows.front();
  }
};

// The instantiated kernels for frames of H x W, or nullptr.
const FixedShape* find_fixed(int H, int W);

// whether the row kernels chosen for `ppb` pairs per block tile H/2 row pairs exactly
bool fixed_supports(const FixedShape& fs, int H, int ppb);

// row forward, column pass, row inverse and finalisation of one wave (a.nitems candidates)
void launch_fixed_wave(const PassArgs& a, const FixedShape& fs, int col_variant, cudaStream_t s, LaunchCounter& lc);

// every phase of p.G candidates (items 0..G-1 of a) in one persistent launch;
// a.spec / a.stats hold p.S workspace slots
void launch_persistent(const PassArgs& a, const PersistArgs& p, const FixedShape& fs, int sm_count, cudaStream_t s,
                       LaunchCounter& lc);

constexpr int kPersistSlots = 8;

// TMA descriptors (CUtensorMap, 128 bytes each) of a fingerprint spectrum
// [H][W/2] (float2 for kF32, __half2 for kF16) for column strips of 2, 4, 8
// and 16 columns, written to host memory `out` (4 descriptors).  False when
// the frame size has no compile-time-planned kernels or the driver lacks TMA.
bool encode_fp_tmaps(const void* spec, int dtype, int H, int W, void* out);
constexpr size_t kFpTmapBytes = 4 * 128;

}  // namespace prnu
