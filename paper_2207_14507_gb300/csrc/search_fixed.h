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

// one instantiated pair of row kernels: row pairs per block, threads per pair
struct FixedRow {
  int ppb;
  int threads;
  size_t smem;
  void* fwd[3];              // by residual storage type
  void* inv;
};

struct FixedShape {
  int W, H;
  std::vector<FixedRow> rows;
  std::vector<FixedCol> cols;
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

// row forward, column pass and row inverse of one wave (a.nitems candidates)
void launch_fixed_wave(const PassArgs& a, const FixedShape& fs, int col_variant, cudaStream_t s, LaunchCounter& lc);

}  // namespace prnu
