// noalloc.cu -- pce_score_noalloc: the aligned-pair PCE of pce_score for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs where the allocator is
// off limits (a real-time or embedded pipeline that fixes its memory at
// start-up, a host framework that owns every device allocation, a process
// that has already used its whole memory budget).  This entry point needs no
// context and no fingerprint handle and allocates nothing: its scratch is the
// file-scope array below, which every GPU that loads the library holds until
// the process exits.
//
// Limits and rules:
//  - frames of at most kMaxPixels = 2^20 pixels (for example 1280x720 or
//    1024x1024), each side at most 4096, under the same size rule as pce_score;
//    larger frames are rejected with PRNU_EINVAL;
//  - every call shares the one scratch array and leaves its contents behind;
//    calls whose GPU work overlaps (two streams, two host threads) race on it,
//    so callers must order them, for example on one stream;
//  - the first call on a device looks up the array's device address
//    (cudaGetSymbolAddress) and sets the kernels' shared-memory limits; make
//    that first call before any stream capture on the device.
#include <math.h>
#include <string.h>

#include <mutex>

#include "internal.h"

namespace prnu {

namespace {

constexpr int kMaxPixels = 1 << 20;
constexpr int kMaxSide = 4096;
constexpr int kNblk = 256;

// Scratch layout (bytes): two packed half spectra, row statistics, twiddles
// for the two FFT lengths, descriptors, fingerprint statistics.
constexpr size_t kSpecBytes = (size_t)kMaxPixels / 2 * sizeof(float2);
constexpr size_t kOffSpecX = 0;
constexpr size_t kOffSpecK = kOffSpecX + kSpecBytes;
constexpr size_t kOffStats = kOffSpecK + kSpecBytes;
constexpr size_t kOffTw = kOffStats + (size_t)kMaxSide * sizeof(RowStat);
constexpr size_t kOffItem = kOffTw + 2 * (size_t)kMaxSide * sizeof(float2);
constexpr size_t kOffFp = kOffItem + 256;
constexpr size_t kOffResult = kOffFp + 256;
constexpr size_t kOffScal = kOffResult + 256;
constexpr size_t kOffPartials = kOffScal + 256;
constexpr size_t kScratchBytes = kOffPartials + 2 * kNblk * sizeof(double);

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// w_n^k = exp(-2 pi i k / n), evaluated in double and rounded to float
__global__ void k_noalloc_twiddles(float2* __restrict__ tw, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)k / (double)n, &s, &c);
    tw[k] = make_float2((float)c, (float)(-s));
  }
}

__global__ void k_noalloc_descriptors(WorkItem it, FpDesc fd, WorkItem* __restrict__ dit, FpDesc* __restrict__ dfd) {
  *dit = it;
  *dfd = fd;
}

unsigned char* scratch_for_device(int dev) {
  if (dev < 0 || dev >= kMaxDevices) throw Error{PRNU_EINVAL, "device index out of range"};
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess)
      throw Error{PRNU_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e)};
    set_kernel_attributes();
    g_addr[dev] = reinterpret_cast<unsigned char*>(p);
  }
  return g_addr[dev];
}

// PRNU_EINVAL unless p is device memory of device `dev`
void check_device_pointer(const void* p, int dev, const char* what) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    throw Error{PRNU_EINVAL, std::string(what) + " is not a CUDA pointer"};
  }
  if (at.type != cudaMemoryTypeDevice || at.device != dev)
    throw Error{PRNU_EINVAL, std::string(what) + " must be device memory of the current device (" +
                                 std::to_string(dev) + ")"};
}

}  // namespace

}  // namespace prnu

using namespace prnu;

extern "C" int pce_score_noalloc(const float* d_X, const float* d_K, int H, int W, double* pce, int* dy, int* dx,
                                 float* peak, prnu_stream stream) {
  try {
    PRNU_CHECK_ARG(d_X && d_K, "NULL argument");
    validate_shape(H, W);
    PRNU_CHECK_ARG((long long)H * W <= kMaxPixels,
                   "pce_score_noalloc takes at most 2^20 pixels (" + std::to_string(H) + "x" + std::to_string(W) +
                       " given); use pce_score for larger frames");
    int dev = 0;
    PRNU_CUDA_TRY(cudaGetDevice(&dev));
    // both images must be device memory of the current device: the kernels
    // below read H*W floats through each pointer on this device
    check_device_pointer(d_X, dev, "X");
    check_device_pointer(d_K, dev, "K");
    unsigned char* base = scratch_for_device(dev);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    LaunchCounter lc;

    float2* specX = reinterpret_cast<float2*>(base + kOffSpecX);
    float2* specK = reinterpret_cast<float2*>(base + kOffSpecK);
    RowStat* stats = reinterpret_cast<RowStat*>(base + kOffStats);
    float2* tw = reinterpret_cast<float2*>(base + kOffTw);
    WorkItem* ditem = reinterpret_cast<WorkItem*>(base + kOffItem);
    FpDesc* dfp = reinterpret_cast<FpDesc*>(base + kOffFp);
    CandResult* dres = reinterpret_cast<CandResult*>(base + kOffResult);
    float* scal = reinterpret_cast<float*>(base + kOffScal);   // mean, scale, inv_scale
    double* partials = reinterpret_cast<double*>(base + kOffPartials);

    // twiddle tables: length W at tw[0], length H at tw[kMaxSide] (the
    // offsets are set here, not looked up, so H == W needs no special case)
    const std::vector<int> zero_off(kMaxFft + 1, 0);
    FftPlan prow = make_plan(W, zero_off);
    FftPlan pcol = make_plan(H, zero_off);
    prow.tw_off = 0;
    pcol.tw_off = kMaxSide;
    k_noalloc_twiddles<<<8, 256, 0, s>>>(tw, W);
    PRNU_CUDA_TRY(cudaGetLastError());
    k_noalloc_twiddles<<<8, 256, 0, s>>>(tw + kMaxSide, H);
    PRNU_CUDA_TRY(cudaGetLastError());

    WorkItem it{};
    it.a11 = it.a22 = 1.f;
    it.lam = 1.f;
    FpDesc fd{specK, kF32, scal + 2};
    k_noalloc_descriptors<<<1, 1, 0, s>>>(it, fd, ditem, dfp);
    PRNU_CUDA_TRY(cudaGetLastError());

    int rowT, rowMB;
    row_launch_shape(prow, &rowT, &rowMB);
    int lg = 0;
    for (int k = 4; k >= 0; --k)
      if (2 * (size_t)H * (1u << k) * sizeof(float2) <= 112 * 1024) {
        lg = k;
        break;
      }
    PassArgs a{};
    a.rdtype = kF32;
    a.H = H;
    a.W = W;
    a.items = ditem;
    a.item0 = 0;
    a.nitems = 1;
    a.stats = stats;
    a.results = dres;
    a.fps = dfp;
    a.tw = tw;
    a.prow = prow;
    a.pcol = pcol;
    a.pairs_per_block = 2;
    a.col_log2 = lg;
    a.row_threads = rowT;

    // fingerprint term: spectrum of K - mean(K), FP32.  Its row spectrum goes
    // to specX (free until X's row pass) so that the column pass reads one
    // buffer and writes another.
    launch_fp_stats(d_K, H, W, partials, kNblk, scal, scal + 1, scal + 2, false, s, lc);
    a.resid = d_K;
    a.spec = specX;
    launch_row_forward(a, false, scal, nullptr, s, lc);
    launch_col(a, 1, specK, nullptr, scal + 1, s, lc);
    // the pair: row FFT of X, correlation with the fingerprint, PCE
    a.resid = d_X;
    a.spec = specX;
    launch_row_forward(a, false, nullptr, nullptr, s, lc);
    launch_col(a, 0, nullptr, nullptr, nullptr, s, lc);
    launch_row_inverse(a, nullptr, s, lc);
    launch_finalize(a, s, lc);

    CandResult r{};
    PRNU_CUDA_TRY(cudaMemcpyAsync(&r, dres, sizeof(CandResult), cudaMemcpyDeviceToHost, s));
    PRNU_CUDA_TRY(cudaStreamSynchronize(s));
    if (pce) *pce = r.pce;
    if (dy) *dy = r.py < H / 2 ? r.py : r.py - H;
    if (dx) *dx = r.px < W / 2 ? r.px : r.px - W;
    if (peak) *peak = r.peak;
    set_error("");
    return PRNU_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.code;
  } catch (const std::exception& e) {
    set_error(e.what());
    return PRNU_EINVAL;
  }
}
