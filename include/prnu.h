/*
 * prnu.h -- C ABI of libprnu: GPU grid search that inverts electronic image
 * stabilisation (EIS) before PRNU camera-fingerprint matching, after
 * "GPU-accelerated SIFT-aided source identification of stabilized videos"
 * (arXiv 2207.14507).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns an int status (PRNU_OK == 0).  Nothing throws
 *    across the ABI.  On failure, prnu_last_error() gives a thread-local
 *    message and no output is written.
 *  - "d_" pointers are device pointers owned by the caller (for example
 *    allocated by PyTorch); they must stay valid until the work enqueued on
 *    the given stream has completed.  The library owns only its context, its
 *    fingerprint-spectrum cache, its scratch workspace and its serving buffers.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued on it in order.  Calls on one context are
 *    serialised by the library (one workspace per context); work from a call on
 *    another stream is ordered after the previous call's work by an event.
 *  - Images are row-major, [rows H][columns W]; a frame batch is [F][H][W].
 *  - Sizes accepted by the correlation path: H and W even, 16 <= H, W <= 4096,
 *    and both 5-smooth (only prime factors 2, 3, 5).  Other sizes return
 *    PRNU_EINVAL.
 *  - Shifts are cyclic and reported signed: dy in [-H/2, H/2), dx in [-W/2, W/2).
 */
#ifndef PRNU_H
#define PRNU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
enum {
    PRNU_OK = 0,
    PRNU_EINVAL = 1,          /* bad argument (size, pointer, window outside the grid) */
    PRNU_ENOMEM = 2,          /* allocation failed or the HBM budget would be exceeded */
    PRNU_ECUDA = 3,           /* a CUDA runtime call failed */
    PRNU_EAGAIN = 4,          /* not ready yet (query_poll with timeout 0), or queue full */
    PRNU_ETIMEOUT = 5,        /* query_poll waited timeout_us and the query is not done */
    PRNU_ENOTFOUND = 6,       /* unknown fingerprint handle or query id */
    PRNU_EDEVICE_ABORT = 7    /* a bounded device-side wait gave up */
};

/* storage types of residuals and fingerprint spectra (arithmetic is always FP32) */
enum { PRNU_F32 = 0, PRNU_F16 = 1, PRNU_BF16 = 2 };

/* prnu_residual flags */
enum {
    PRNU_WEIGHT_BY_INTENSITY = 1, /* store R = I * W(I) (the K.I matching term) instead of W(I) */
    PRNU_NORMALISE = 2            /* scale each frame's R by 1/RMS(R) (s = 1 for R == 0) */
};

typedef struct prnu_ctx prnu_ctx;
typedef void* prnu_stream;          /* a cudaStream_t */

/* Search grid: lambda_i = lam0 + i*dlam (0 <= i < nlam), theta_j = th0_deg + j*dth_deg
 * degrees (0 <= j < nth).  Node values are evaluated in double from these float
 * fields and rounded to float.  Candidate index = i*nth + j (lambda-major).
 * Sec. 3.2 ("correction", Eq. 8): exhaustive search over Lambda x Theta. */
typedef struct {
    float lam0, dlam;
    int nlam;
    float th0_deg, dth_deg;
    int nth;
} prnu_grid;

/* Inclusive index window of one frame: lam_lo..lam_hi x th_lo..th_hi. */
typedef struct {
    int lam_lo, lam_hi, th_lo, th_hi;
} prnu_window;

/* Best candidate of one (frame, fingerprint) pair. */
typedef struct {
    float lam, th_deg;      /* arg-max scale and rotation (degrees) */
    int dy, dx;             /* arg-max cyclic shift, signed */
    double pce;             /* Eq. 3 at the arg-max */
    float peak;             /* correlation value at the peak, C* = sum_x X(x) K0(x + d*) */
    int cand_idx;           /* i*nth + j, or -1 when the frame had no candidate */
} prnu_result;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device
 * memory the library itself allocates (workspace, spectra cache, serving
 * buffers); 0 means 90% of the free memory at creation.  *out receives the
 * context.  Errors: PRNU_EINVAL (NULL out, bad device), PRNU_ECUDA. */
int prnu_create(prnu_ctx** out, int device, size_t hbm_budget_bytes);

/* Wait for outstanding work, stop the serving thread, free everything the
 * context owns.  NULL is accepted. */
int prnu_destroy(prnu_ctx* ctx);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* prnu_last_error(void);

/* Number of CUDA kernels this context has launched so far. */
uint64_t prnu_launch_count(const prnu_ctx* ctx);

/* ---------------------------------------------------------------- hot path */

/* Noise residual of F uint8 frames (Sec. 2.2: W(I) = I - F(I)), with F a 3x3
 * local Wiener filter: local mean mu and population variance s2 over the 3x3
 * neighbourhood (borders replicated), noise power nu2 = mean of s2 over the
 * frame, Wiener(I) = mu + (I - mu) max(s2 - nu2, 0) / max(s2, nu2).
 *  d_frames: device uint8, frame f row y at d_frames + (f*H + y)*pitch, pitch >= W.
 *  flags:    PRNU_WEIGHT_BY_INTENSITY and/or PRNU_NORMALISE.
 *  out_dtype: PRNU_F32 | PRNU_F16 | PRNU_BF16; d_out: [F][H][W] of that type.
 *  d_scale:  [F] float, receives the per-frame scale s (1 without PRNU_NORMALISE);
 *            may be NULL.
 * H, W >= 1 (no FFT-size rule here).  F == 0 is a no-op.  Asynchronous. */
int prnu_residual(prnu_ctx* ctx, const uint8_t* d_frames, int F, int H, int W, size_t pitch,
                  int flags, int out_dtype, void* d_out, float* d_scale, prnu_stream stream);

/* Reference fingerprint of a device from L of its frames (Eq. 2):
 *     K = (sum_l I_l * W(I_l)) / (sum_l I_l * I_l),   every operation pixel-wise,
 * W the residual of prnu_residual (3x3 Wiener, per-frame noise power); 0 where
 * every frame is 0.  Sums in double; frames are taken 16 at a time.
 *  d_frames: device uint8, frame l row y at d_frames + (l*H + y)*pitch, pitch >= W
 *            (0 means W).
 *  d_K:      device float [H][W], written.
 * H, W >= 1, L >= 1.  Asynchronous on `stream`.
 * Errors: PRNU_EINVAL (sizes, NULL), PRNU_ENOMEM (workspace over the budget). */
int prnu_fingerprint_estimate(prnu_ctx* ctx, const uint8_t* d_frames, int L, int H, int W, size_t pitch,
                              float* d_K, prnu_stream stream);

/* Fingerprint term (Eq. 1-3): cache the 2-D spectrum of K0 = K - mean(K) on the
 * device, in the library's packed half-spectrum layout, stored as FP32 or FP16
 * (store_dtype PRNU_F32 | PRNU_F16; PRNU_BF16 is stored as FP16).  d_K: device
 * float [H][W].  *out_handle receives a reference-counted handle; computing
 * the same device buffer twice gives two handles.  The spectrum is complete
 * when the work on `stream` is; later calls on any stream are ordered after it.
 * Errors: PRNU_EINVAL (size rule), PRNU_ENOMEM (budget). */
int prnu_fingerprint_term(prnu_ctx* ctx, const float* d_K, int H, int W, int store_dtype,
                          uint64_t* out_handle, prnu_stream stream);

/* Drop a handle's reference; the cached spectrum is freed with the last one.
 * Errors: PRNU_ENOTFOUND. */
int prnu_fingerprint_release(prnu_ctx* ctx, uint64_t handle);

/* EIS inversion grid search (Sec. 3.2 "correction" over one grid level, Eq. 3
 * scoring, Eq. 4 restricted to scale + rotation).  For every frame f, every
 * fingerprint p and every candidate (lambda_i, theta_j) in the frame's window:
 *   X(p) = bilinear(R_f, c + Rot(-theta)(p - c)/lambda), c = ((W-1)/2, (H-1)/2),
 *          taps outside the frame count 0;
 *   C(d) = sum_x X(x) K0_p((x + d) mod (H, W))  over all H*W cyclic shifts;
 *   PCE  = sgn(C*) C*^2 / E, C* = max C (first in row-major order on ties),
 *          E = mean of C^2 outside the cyclic 11x11 window around the peak
 *          (E == 0: PCE = 0 for a zero peak, +-inf otherwise);
 * then keeps, per (f, p), the candidate of largest PCE (ties: lowest index).
 *  d_resid:  [F][H][W] residuals of type `dtype` (from prnu_residual).
 *  d_scale:  [F] or NULL; when given, the reported peak is divided by d_scale[f].
 *  fp_handles: host array [P] of handles of spectra of the same H x W.
 *  grid:     host pointer.  windows: host array [F] or NULL (= full grid).
 *  out:      [F*P] results, out[f*P + p]; host or device pointer.  With a host
 *            pointer the call returns after the stream has finished; with a
 *            device pointer it is asynchronous.
 *  d_all_pce: device double [F*P*nlam*nth] or NULL; receives every evaluated
 *            candidate's PCE at (f*P + p)*nlam*nth + cand_idx, NaN elsewhere.
 * With P > 1 the candidates of one frame and node share the warp, the row FFT
 * and the forward column FFT (they do not depend on the fingerprint), on the
 * sizes with compile-time-planned kernels, unless prnu_tuning.share_forward
 * is 0; the results are the same bit for bit either way.
 * F == 0 or P == 0 is a no-op.  Errors: PRNU_EINVAL, PRNU_ENOTFOUND, PRNU_ENOMEM. */
int eis_grid_search(prnu_ctx* ctx, const void* d_resid, int dtype, const float* d_scale,
                    int F, int H, int W, const uint64_t* fp_handles, int P,
                    const prnu_grid* grid, const prnu_window* windows,
                    prnu_result* out, double* d_all_pce, prnu_stream stream);

/* The same search through the plain per-candidate path: one candidate at a
 * time, each step (warp, row FFT, column FFT, spectrum product, inverse column
 * FFT, inverse row FFT, PCE) its own launch through full-size FP32
 * intermediates in device memory.  Same arguments and results as
 * eis_grid_search (dtype must be PRNU_F32); it exists as the speed baseline. */
int eis_grid_search_naive(prnu_ctx* ctx, const void* d_resid, int dtype, const float* d_scale,
                          int F, int H, int W, const uint64_t* fp_handles, int P,
                          const prnu_grid* grid, const prnu_window* windows,
                          prnu_result* out, double* d_all_pce, prnu_stream stream);

/* Noise residual by Mihcak's wavelet denoiser (the paper's denoiser, Sec.
 * 2.2), the alternative to prnu_residual's 3x3 Wiener filter, with the same
 * arguments plus the noise level sigma0 (grey levels; 3 is a common choice):
 *   - the frame mirrored at its bottom and right edges (half-sample) up to
 *     multiples of 16;
 *   - a 4-level orthonormal separable transform with Daubechies' 8-tap filter
 *     (4 vanishing moments), periodic;
 *   - every detail coefficient c replaced by its noise part
 *     c sigma0^2 / (s2 + sigma0^2), s2 = the smallest over W in {3, 5, 7, 9}
 *     of max(0, mean of c^2 over the W x W window of its band - sigma0^2)
 *     (zeros outside the band; 0 where s2 + sigma0^2 = 0); the coarsest
 *     approximation band replaced by 0;
 *   - the inverse transform cropped to H x W: W(I) = I - F(I);
 *     R = I W(I) with PRNU_WEIGHT_BY_INTENSITY, else W(I); PRNU_NORMALISE as
 *     prnu_residual.
 * FP32 arithmetic.  H, W >= 16.  Scratch: two (H, W rounded up to 16) float
 * images per frame, up to 16 frames at a time within a quarter of what the
 * HBM budget leaves.  Asynchronous.  PRNU_EINVAL for a negative or
 * non-finite sigma0, frames below 16 x 16, unknown flags. */
int prnu_residual_wavelet(prnu_ctx* ctx, const uint8_t* d_frames, int F, int H, int W, size_t pitch, int flags,
                          int out_dtype, double sigma0, void* d_out, float* d_scale, prnu_stream stream);

/* The reference fingerprint brought to a video's geometry: down-scaled (or
 * up-scaled) by `scale` and cropped (Sec. 3: the fingerprint estimated from
 * images must be down-scaled and cropped before it tests video frames; the
 * paper gives no resampling, this is the antialiased bilinear one).  Output
 * sample o of an axis sits at input position u = (o + first + 0.5)/scale - 0.5;
 * its weights are the tent max(0, 1 - |j - u| a), a = min(scale, 1) (widened by
 * 1/scale when shrinking), normalised, indices beyond the ends replicated;
 * rows and columns separably.
 *  d_Kin:  device float [Hin][Win], row pitch in_pitch elements (0 = Win).
 *  scale:  in [1/64, 64]; the resized fingerprint has round(Hin*scale) x
 *          round(Win*scale) samples.
 *  y0, x0: top-left of the crop in the resized fingerprint; the H x W crop
 *          must lie inside it.
 *  d_Kout: device float [H][W] (dense), may not overlap d_Kin.
 * FP32 accumulation of FP32 weights computed in double.  Synchronous.
 * PRNU_EINVAL for a scale or crop out of range. */
int prnu_fingerprint_resize(prnu_ctx* ctx, const float* d_Kin, int Hin, int Win, size_t in_pitch, double scale,
                            int y0, int x0, float* d_Kout, int H, int W, prnu_stream stream);

/* The grid search as Sec. 3.2 literally states it: for every candidate the
 * FRAME is warped and the residual is extracted from the warped frame, instead
 * of warping a residual computed once per frame (eis_grid_search).  For frame f
 * and candidate (lambda, theta):
 *     X(p) = bilinear(I_f, c + Rot(-theta)(p - c) / lambda), taps outside 0,
 *     W(X) = X - Wiener3x3(X) (3x3 moments, borders replicated, noise power
 *            the mean local variance of X), R = X * W(X) with
 *            PRNU_WEIGHT_BY_INTENSITY, else R = W(X) (the plain Eq. 3 term),
 * then R is correlated with the fingerprint and scored by PCE as in
 * eis_grid_search (identity warp).  Every candidate costs one more pass over
 * the frame than eis_grid_search.
 *  d_frames: device uint8 [F][H][W], row pitch `pitch` bytes (0 = W).
 *  flags:    0 or PRNU_WEIGHT_BY_INTENSITY.
 *  fp_handles, P, grid, windows: as eis_grid_search.
 *  out:      prnu_result [F*P], host or device memory.
 * FP32 arithmetic and storage.  Synchronous (waits for `stream`).  Errors as
 * eis_grid_search; PRNU_EINVAL for other flags. */
int eis_grid_search_frames(prnu_ctx* ctx, const uint8_t* d_frames, int F, int H, int W, size_t pitch, int flags,
                           const uint64_t* fp_handles, int P, const prnu_grid* grid, const prnu_window* windows,
                           prnu_result* out, prnu_stream stream);

/* The correction operator of Sec. 3.2: for every (frame f, fingerprint p)
 * pair a breadth-first search over (lambda, theta) that maximises the PCE.
 * Iteration n (1-based) searches, around the previous estimate
 * (lambda(n-1), theta(n-1)), the nodes
 *     lambda(n-1) + a * 0.01 * 10^-(n-1),        a in -5..5,
 *     theta(n-1)  + b * 0.1 * 10^-(n-1) degrees, b in -5..5
 *     (b in -th_half1..th_half1 at n = 1: the text's denser first angle grid,
 *      -5..5 degrees in steps of 0.1 for th_half1 = 50),
 * each node the float32 rounding of the double sum centre + a * float32(step);
 * that is the reading of Eq. 8, whose printed steps 0.01^-n and 0.1^-n would
 * widen the neighbourhoods.  An iteration keeps its node of highest PCE (ties
 * to the lowest index, scale-major); the search stops when that node is its
 * centre (the estimate did not change) or after max_iter iterations, and
 * returns the best PCE seen over all iterations (the earliest on ties).
 * Every iteration runs the hot path of eis_grid_search over all pairs still
 * searching.
 *  d_resid, dtype, d_scale, F, H, W, fp_handles, P: as eis_grid_search.
 *  init_lam, init_th: host float [F*P] start estimates (index f*P + p), or NULL
 *      for lambda(0) = 1 and theta(0) = 0.
 *  max_iter >= 1 (the paper uses 3); th_half1 >= 0 (0 selects 50).
 *  out:   host prnu_result [F*P]: the best node (lam, th_deg, shift, PCE);
 *         cand_idx = a'*nb + b' within the node grid of the iteration that
 *         found it (a', b' >= 0, nb = 2*th_half1 + 1 at n = 1, else 11).
 *  iters: host int [F*P], iterations run per pair, or NULL.
 * Synchronous (waits for `stream`).  Errors as eis_grid_search. */
int eis_correction(prnu_ctx* ctx, const void* d_resid, int dtype, const float* d_scale, int F, int H, int W,
                   const uint64_t* fp_handles, int P, const float* init_lam, const float* init_th,
                   int max_iter, int th_half1, prnu_result* out, int* iters, prnu_stream stream);

/* (lambda, theta) of the similarity nearest to a homography's linear part: the
 * start estimate the correction takes from a co-registration (Sec. 3.2, "a
 * vector t_init is derived").  Hm: host double [3][3], row-major, acting on
 * (x = column, y = row, 1) so that the registered frame is H applied to the
 * frame; with M = the upper-left 2x2 of Hm / Hm[2][2],
 *     a = (m00 + m11) / 2,  b = (m10 - m01) / 2,
 *     lambda = hypot(a, b),  theta = atan2(b, a) in degrees,
 * the least-squares fit of lambda * Rot(theta).  The translation and the
 * projective terms are dropped, as the correction assumes (Sec. 3.2).  This is
 * the convention of the correction's warp: the node (lambda, theta) maps the
 * frame forward by lambda * Rot(theta) about the frame centre.
 * PRNU_EINVAL for a non-finite entry, Hm[2][2] == 0 or a zero linear part. */
int similarity_from_homography(const double* Hm, float* lam, float* th_deg);

/* Algorithm 1 (SIFT-aided EIS inversion) with the co-registration supplied by
 * the caller, and the decision of Sec. 3.2: for a segment of F frames
 * (frame 0 the anchor I_A, frames 1..F-1 the successive P_v) and one
 * fingerprint,
 *   - the anchor is corrected from (1, 0);
 *   - frame v >= 1 is scored unwarped (the node (1, 0)) and co-registered (the
 *     node similarity_from_homography(H_v)); the correction starts from the
 *     co-registration if that PCE is strictly higher, else from (1, 0);
 *   - gamma[v] = the highest PCE its correction found;
 *   - the decision is mean(gamma) > tau (the paper's tau = 19.5 is set for a
 *     false-positive rate of about 0.05 on its 1080p videos, Table 1).
 * H_v co-registers P_v with the corrected previous frame (the paper's
 * coregistration operator, SIFT keypoints and DEGENSAC: host-side, not in this
 * library; the caller builds the corrected frame from best[v-1]).  Given every
 * H_v the frames are independent, so both PCE tests run as one batched search
 * and the corrections as one batched correction.  The registered frame's PCE
 * uses the similarity part of H_v only: its translation moves the correlation
 * peak, which the search over all cyclic shifts finds anyway.
 *  d_resid, dtype, d_scale, H, W: as eis_grid_search, F >= 1 frames.
 *  fp_handle:    the reference fingerprint (size H x W).
 *  homographies: host double [F][3][3] row-major (entry 0 unused), or NULL to
 *                start every frame from (1, 0).
 *  max_iter, th_half1: as eis_correction (the paper: 3 and 50).
 *  gamma:      host double [F], the PCE vector.
 *  mean_gamma: host double, or NULL.  decision: host int (1 = the video comes
 *              from the fingerprint's camera), or NULL.
 *  best:       host prnu_result [F] (the node of gamma[v]), or NULL.
 *  from_reg:   host int [F], 1 where the correction started from H_v, or NULL.
 * Synchronous (waits for `stream`).  Errors as eis_correction, plus
 * PRNU_EINVAL for a homography similarity_from_homography rejects. */
int eis_invert_video(prnu_ctx* ctx, const void* d_resid, int dtype, const float* d_scale, int F, int H, int W,
                     uint64_t fp_handle, const double* homographies, int max_iter, int th_half1, double tau,
                     double* gamma, double* mean_gamma, int* decision, prnu_result* best, int* from_reg,
                     prnu_stream stream);

/* PCE of one aligned pair (Eq. 3, no warp): d_X device float [H][W] against the
 * cached fingerprint `fp_handle`.  Host outputs; any of them may be NULL.
 * Synchronous (waits for `stream`). */
int pce_score(prnu_ctx* ctx, const float* d_X, uint64_t fp_handle, int H, int W,
              double* pce, int* dy, int* dx, float* peak, prnu_stream stream);

/* pce_score for callers that cannot allocate device memory (the paper has no
 * counterpart: this is a deployment variant).  Some callers cannot call
 * cudaMalloc -- code where the allocator is off limits, such as a real-time
 * pipeline that fixes its memory at start-up, a host framework that owns every
 * device allocation, or a process already at its memory budget.  This entry
 * point needs no context and no fingerprint handle and allocates nothing: it
 * computes the PCE of d_X (device float [H][W]) against the fingerprint d_K
 * (device float [H][W], mean removed inside) in a fixed static device scratch
 * array of about 8.5 MB that every GPU loading the library holds until exit.
 *  - H*W must not exceed 2^20 pixels (e.g. 1280x720, 1024x1024), with the
 *    size rule of pce_score; larger frames return PRNU_EINVAL.
 *  - All calls share the scratch array, which keeps the last call's contents;
 *    calls whose GPU work overlaps race on it, so order them (one stream).
 *  - The first call on a device looks up the array's address and sets kernel
 *    attributes; make it before any stream capture on that device.
 *  - d_X and d_K must both be device memory of the current device (checked
 *    with cudaPointerGetAttributes: PRNU_EINVAL otherwise); the caller keeps
 *    them H*W floats long and dense.
 * Host outputs, any of them may be NULL.  Synchronous (waits for `stream`). */
int pce_score_noalloc(const float* d_X, const float* d_K, int H, int W,
                      double* pce, int* dy, int* dx, float* peak, prnu_stream stream);

/* ---------------------------------------------------------------- serving */

/* One forensic query: F frames tested against P fingerprints. */
typedef struct {
    const uint8_t* frames;          /* [F][H][W] uint8 (row pitch `pitch`), device or host memory;
                                       must stay valid until query_poll returns PRNU_OK */
    int F, H, W;
    size_t pitch;                   /* bytes between rows (>= W); 0 means W */
    const uint64_t* fp_handles;     /* [P] spectra handles of size H x W (copied at submit) */
    int P;
    prnu_grid grid;
    const prnu_window* windows;     /* [F] or NULL = full grid (copied at submit) */
    int dtype;                      /* residual storage type */
    int flags;                      /* residual flags (PRNU_WEIGHT_BY_INTENSITY, PRNU_NORMALISE) */
} prnu_query;

/* Hand a query to the context's continuous-batching server.  The descriptor is
 * copied; *qid receives its id.  The server admits queries in arrival order as
 * their device memory fits the context's HBM budget, and interleaves the
 * candidates of all admitted queries in shared launches.
 * Errors: PRNU_EINVAL, PRNU_ENOTFOUND, PRNU_EAGAIN (queue full), PRNU_ENOMEM
 * (the query alone exceeds the budget). */
int query_submit(prnu_ctx* ctx, const prnu_query* q, uint64_t* qid);

/* Wait up to timeout_us microseconds (0 = do not wait, < 0 = forever) for
 * query `qid`.  PRNU_OK: out[F*P] (host) receives the results and the query is
 * retired.  PRNU_EAGAIN (timeout 0) / PRNU_ETIMEOUT: not done yet.
 * PRNU_ENOTFOUND: unknown or already retired id.  Errors inside the server are
 * reported here (PRNU_ECUDA, PRNU_EDEVICE_ABORT). */
int query_poll(prnu_ctx* ctx, uint64_t qid, prnu_result* out, int64_t timeout_us);

/* Latency of a finished query (kept for the last 100000 queries): time from
 * query_submit to admission (queued_ms) and to the moment its results reached
 * host memory (total_ms), in milliseconds.  Errors: PRNU_ENOTFOUND. */
int query_latency(prnu_ctx* ctx, uint64_t qid, double* queued_ms, double* total_ms);

/* Request loop of the server.  PRNU_LOOP_HOST: a host thread forms every
 * wave (its candidate, result and frame tables) and launches its kernels.
 * PRNU_LOOP_DEVICE: for frame sizes with compile-time-planned kernels, the
 * loop runs on the GPU.  One CUDA graph per frame size and storage type
 * repeats, in a WHILE node:
 *  - a scheduler kernel takes the next candidates of the admitted queries
 *    (whole forward units, in admission order) from a host-mapped ring and
 *    builds the wave's tables on the device;
 *  - the wave kernels run, in the branch of a SWITCH node whose grids are
 *    the smallest that fit the wave (shared forward units or not);
 *  - a completion kernel writes the arg-max of each query the wave finished
 *    into host-mapped memory and raises its done flag.
 * The host thread only admits queries (device memory, ingest, one ring entry
 * each).  It relaunches a size's graph when it has drained or used its
 * budget of 32 waves, so sizes take turns.  Other sizes take host waves.
 * Results are bit-identical in both modes; PRNU_LOOP_DEVICE is the default.
 * Set the mode before the context's first query_submit: PRNU_EINVAL
 * afterwards (unless unchanged) or for an unknown mode. */
enum { PRNU_LOOP_HOST = 0, PRNU_LOOP_DEVICE = 1 };
int prnu_server_set_loop(prnu_ctx* ctx, int mode);

/* Serving statistics since creation: completed queries, candidates scored,
 * launches issued by the server (with the device loop: graph launches, plus
 * the ingest kernels), and the peak device bytes admitted. */
typedef struct {
    uint64_t queries_done, candidates_done, server_launches;
    uint64_t admitted_bytes_peak, admitted_bytes_now;
} prnu_server_stats;
int prnu_server_stats_get(prnu_ctx* ctx, prnu_server_stats* out);

/* ---------------------------------------------------------------- tuning */

/* Launch configuration of the fused path for one frame size: columns per
 * column-pass block and row pairs per row block of the generic kernels, the
 * candidates per wave (per-candidate spectra kept in the workspace), and which
 * compile-time-planned column kernel to use where the size has them
 * (1920x1080, 1280x720, 3840x2160, 256x256). */
typedef struct {
    int col_width;        /* 4, 8 or 16 */
    int pairs_per_block;  /* 1, 2 or 4 */
    int wave;             /* candidates in flight, >= 1 (default: up to 1024, with at most
                             16 GB of spectra and a quarter of the context's HBM budget) */
    int variant;          /* compile-time-planned column kernel variant for this size
                             (0.. n-1), or -1 for the generic runtime-plan kernels */
    int persistent;       /* 0: waves, one launch sequence each (default).
                             1: sizes with compile-time-planned kernels run a whole call
                             as one persistent launch that schedules every phase of every
                             candidate as tasks (spectra stay in L2).
                             2: sizes with compile-time-planned kernels run every wave of a
                             call in one CUDA graph launch: a scheduler kernel forms each
                             wave on the device and picks the branch of the graph whose
                             grids fit it (the device-resident loop of the query server,
                             over one run).  Results equal those of 0 bit for bit.
                             eis_correction then runs its whole iteration loop on the
                             device: work lists written, scored (one graph launch each)
                             and updated by kernels, one synchronisation at the end. */
    int streams;          /* 1 or 2: waves of compile-time-planned sizes alternate between
                             the call's stream and a second stream of the context, each
                             with its own half of the workspace, so that one wave's
                             kernels overlap the next wave's (set_tuning: 0 keeps 1) */
    int share_forward;    /* 1 (default): with P > 1 fingerprints, the candidates of one
                             frame and grid node (Eq. 3 against each fingerprint) share
                             one warp, row FFT and forward column FFT; the product and the
                             inverse FFT run per fingerprint (compile-time-planned sizes,
                             waves; the results equal those of 0 bit for bit).  0: every
                             candidate runs its own forward pass. */
} prnu_tuning;

/* Read / override the configuration used for frames of H x W. */
int prnu_get_tuning(prnu_ctx* ctx, int H, int W, prnu_tuning* out);
int prnu_set_tuning(prnu_ctx* ctx, int H, int W, const prnu_tuning* cfg);

/* Time the candidate configurations on synthetic data of H x W and `dtype`,
 * keep the fastest for that size and write it to *best (may be NULL).
 * `budget_ms` bounds the total measuring time. */
int prnu_autotune(prnu_ctx* ctx, int H, int W, int dtype, double budget_ms, prnu_tuning* best,
                  prnu_stream stream);

/* ---------------------------------------------------------------- profiling */

/* Per-kernel timing: while a profile is open, every launch of the context is
 * bracketed by two CUDA events recorded on its launching stream. */
typedef struct {
    char name[32];          /* kernel kind, e.g. "row_forward", "column" */
    uint64_t launches;
    double total_ms;        /* sum of the event-measured durations */
} prnu_kernel_stat;

/* Start recording (clears earlier records). */
int prnu_profile_begin(prnu_ctx* ctx);

/* Stop recording, wait for the recorded events and aggregate them by kernel
 * kind into out[0..max) (max >= 1); *n_out receives the number of kinds seen. */
int prnu_profile_end(prnu_ctx* ctx, prnu_kernel_stat* out, int max, int* n_out);

/* ---------------------------------------------------------------- failure injection (tests) */

/* Test hook; the paper has no counterpart.  With key
 * PRNU_DEBUG_STALL_DEVICE_WAITS and value 1, every bounded device-side wait of
 * the compile-time-planned kernels (the column pass's TMA barrier, the
 * persistent kernel's dependency counts) waits for one arrival more than will
 * ever come: each such wait runs out (about a second), the kernel raises the
 * context's device error flag and abandons its candidate, the results of that
 * call are undefined, and the next search call on the context fails with
 * PRNU_EDEVICE_ABORT.  The context stays usable.  Value 0 turns it off.
 * Errors: PRNU_EINVAL (NULL context, unknown key). */
enum { PRNU_DEBUG_STALL_DEVICE_WAITS = 1 };
int prnu_debug_set(prnu_ctx* ctx, int key, int value);

#ifdef __cplusplus
}
#endif
#endif /* PRNU_H */
