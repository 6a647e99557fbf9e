// common.cuh -- structures shared by the kernels and the host side of libprnu.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft.cuh"

namespace prnu {

enum StoreType { kF32 = 0, kF16 = 1, kBF16 = 2 };
// Zero-bordered residual layouts of the compile-time-planned row kernels for
// half storage: element x holds the pair (R[x], R[x + 1]) as one 4-byte
// word, so a bilinear sample takes one aligned load per row.
enum PairStoreType { kF16P = 3, kBF16P = 4 };
constexpr int kNumStoreLayouts = 5;

// One candidate of the search: which frame, which fingerprint, which grid
// node, where its result goes, and the inverse-warp matrix
// q = c + A (p - c), A = Rot(-theta)/lambda (Eq. 4 restricted to a similarity).
struct WorkItem {
  int frame;
  int fp;        // index into the call's fingerprint table
  int cand;      // grid index i*nth + j
  int group;     // (frame, fingerprint) pair index, f*P + p
  float a11, a12, a21, a22;
  float lam, th_deg;
};

// Fingerprint spectrum as the kernels see it.
struct FpDesc {
  const void* spec;    // packed [H][W/2] complex, float2 or __half2
  int dtype;                 // kF32 or kF16
  const float* inv_scale;    // device scalar: multiply the correlation by it to undo the storage scale
  const void* tmaps;         // device CUtensorMap[4] of the spectrum (strips of 2, 4, 8, 16 columns), or nullptr
};

// Per-row statistics of one candidate's correlation surface.
struct RowStat {
  float max;
  int arg;             // column of the first maximum
  double sumsq;        // sum of C^2 over the row
};

// Per-candidate score.
struct CandResult {
  double pce;
  float peak;          // C* in the residual's stored units (FFT scale removed)
  int py, px;          // cyclic peak position
  int cand;
  int group;
  int pad;
};

// Host-built description of one launch of the fused path.
struct PassArgs {
  const void* resid;          // frames of `rdtype`: pixel (y, x) of frame f at f*fpitch + roff + y*rpitch + x
  int rdtype;
  int rpitch;                 // row pitch (elements)
  size_t fpitch;              // frame pitch (elements)
  size_t roff;                // offset of pixel (0, 0) inside a frame (elements)
  int H, W;
  const WorkItem* items;      // all items of the call
  int item0;                  // first item of this wave
  int nitems;                 // items in this wave
  float2* spec;               // workspace spectra [wave][H][W/2]
  RowStat* stats;             // [wave][H]
  CandResult* results;        // [all items]
  const FpDesc* fps;          // [P]
  const float* scale;         // [F] or nullptr
  const float2* tw;           // twiddle table
  FftPlan prow, pcol;
  int pairs_per_block;
  int col_log2;               // columns per column-pass block = 1 << col_log2
  int row_threads;            // threads per row FFT
  // Optional per-slot indirection, used when one wave mixes candidates of
  // several queries (serving): item and result of slot s live at
  // item_ptrs[s] / result_ptrs[s], and frame f's residual at frame_ptrs[f].
  // nullptr = the contiguous arrays above.
  const WorkItem* const* item_ptrs;
  CandResult* const* result_ptrs;
  const void* const* frame_ptrs;
  int* err;                   // device flag set when a bounded device-side wait gives up (may be nullptr)
  int stall;                  // test hook: 1 = every bounded wait expects one arrival too many
  // Forward units: items that share a frame and a grid node and differ only in
  // the fingerprint share one warp, row FFT and forward column FFT, computed
  // in slot nitems + u of the workspace (after the items' slots).  Unit u of
  // the wave holds slots units[u] .. units[u+1]-1 and slot s belongs to unit
  // unit_of[s] (device arrays), or, with units == nullptr, slots u*share ..
  // u*share+share-1.  share = 1 and no table: every item is its own unit and
  // computes in its own slot (nunits == nitems).
  const int* units;
  const int* unit_of;
  int nunits;
  int share;
  // host-side: some fingerprint of the pass is stored FP32 (launch choices only)
  int fp_f32;
  // Device-side counts of a launch whose grid was sized for nitems / nunits
  // slots ahead of time (the query server's device-resident loop): [0] the
  // wave's items, [1] its forward units; blocks past them return at once.
  // nullptr: the grid is exact.
  const int* d_counts;
};

// whether block `b` of a grid over the wave's items (k = 0) or forward units
// (k = 1) lies past the wave's device-side count
__device__ __forceinline__ bool past_count(const PassArgs& a, int b, int k) {
  return a.d_counts != nullptr && b >= __ldcg(a.d_counts + k);
}

__device__ __forceinline__ int unit_first(const PassArgs& a, int u) { return a.units ? a.units[u] : u * a.share; }
__device__ __forceinline__ int unit_of_slot(const PassArgs& a, int s) { return a.unit_of ? a.unit_of[s] : s / a.share; }

__device__ __forceinline__ WorkItem item_of(const PassArgs& a, int slot) {
  return a.item_ptrs ? *a.item_ptrs[slot] : a.items[a.item0 + slot];
}
__device__ __forceinline__ CandResult* result_of(const PassArgs& a, int slot) {
  return a.result_ptrs ? a.result_ptrs[slot] : a.results + a.item0 + slot;
}
// residual of frame f: base pointer, element offset of the frame's pixel (0, 0)
__device__ __forceinline__ const void* frame_of(const PassArgs& a, int f, size_t* base) {
  if (a.frame_ptrs) {
    *base = a.roff;
    return a.frame_ptrs[f];
  }
  *base = (size_t)f * a.fpitch + a.roff;
  return a.resid;
}

// ---------------------------------------------------------------- storage loads / stores

template <int DT>
__device__ __forceinline__ float load_store_type(const void* p, size_t i) {
  if constexpr (DT == kF32) {
    return __ldg(reinterpret_cast<const float*>(p) + i);
  } else if constexpr (DT == kF16) {
    return __half2float(__ldg(reinterpret_cast<const __half*>(p) + i));
  } else {
    return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16*>(p) + i));
  }
}

template <int DT>
__device__ __forceinline__ void store_store_type(void* p, size_t i, float v) {
  if constexpr (DT == kF32) {
    reinterpret_cast<float*>(p)[i] = v;
  } else if constexpr (DT == kF16) {
    reinterpret_cast<__half*>(p)[i] = __float2half_rn(v);
  } else {
    reinterpret_cast<__nv_bfloat16*>(p)[i] = __float2bfloat16_rn(v);
  }
}

__device__ __forceinline__ float2 load_spec(const void* p, int dtype, size_t i) {
  if (dtype == kF32) return __ldg(reinterpret_cast<const float2*>(p) + i);
  __half2 h = reinterpret_cast<const __half2*>(p)[i];
  return __half22float2(h);
}

}  // namespace prnu
