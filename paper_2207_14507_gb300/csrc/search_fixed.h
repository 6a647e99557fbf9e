// search_fixed.h -- registry of the compile-time-planned kernels (search_fixed.cu).
#pragma once
#include <vector>

#include "internal.h"

namespace prnu {

// one instantiated column-pass variant: columns per block, threads, shared memory
struct FixedCol {
  int nc;
  int threads;
  size_t smem;
  void* fn;
};

struct FixedShape {
  int W, H;
  int row_threads, ppb;
  size_t row_smem;
  void* row_fwd[3];          // by residual storage type
  void* row_inv;
  std::vector<FixedCol> cols;
};

// The instantiated kernels for frames of H x W, or nullptr.
const FixedShape* find_fixed(int H, int W);

// row forward, column pass and row inverse of one wave (a.nitems candidates)
void launch_fixed_wave(const PassArgs& a, const FixedShape& fs, int col_variant, cudaStream_t s, LaunchCounter& lc);

}  // namespace prnu
