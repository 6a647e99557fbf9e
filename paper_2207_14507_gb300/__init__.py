"""Python binding of libprnu (ctypes).  Argument marshalling only: every step of
the search runs in the library's CUDA kernels.  PyTorch supplies device memory
and streams.

The raw C functions are exposed under their C names on ``lib()``; ``Context``
wraps the same calls with tensor arguments (same method names).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libprnu.so")

PRNU_OK, PRNU_EINVAL, PRNU_ENOMEM, PRNU_ECUDA, PRNU_EAGAIN, PRNU_ETIMEOUT, PRNU_ENOTFOUND, PRNU_EDEVICE_ABORT = range(8)
PRNU_F32, PRNU_F16, PRNU_BF16 = 0, 1, 2
PRNU_WEIGHT_BY_INTENSITY, PRNU_NORMALISE = 1, 2
PRNU_DEBUG_STALL_DEVICE_WAITS = 1
PRNU_LOOP_HOST, PRNU_LOOP_DEVICE = 0, 1
STATUS_NAMES = {0: "PRNU_OK", 1: "PRNU_EINVAL", 2: "PRNU_ENOMEM", 3: "PRNU_ECUDA", 4: "PRNU_EAGAIN",
                5: "PRNU_ETIMEOUT", 6: "PRNU_ENOTFOUND", 7: "PRNU_EDEVICE_ABORT"}


class PrnuError(RuntimeError):
    def __init__(self, code: int, func: str, msg: str):
        super().__init__(f"{func}: {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class prnu_grid(C.Structure):
    _fields_ = [("lam0", C.c_float), ("dlam", C.c_float), ("nlam", C.c_int),
                ("th0_deg", C.c_float), ("dth_deg", C.c_float), ("nth", C.c_int)]


class prnu_window(C.Structure):
    _fields_ = [("lam_lo", C.c_int), ("lam_hi", C.c_int), ("th_lo", C.c_int), ("th_hi", C.c_int)]


class prnu_result(C.Structure):
    _fields_ = [("lam", C.c_float), ("th_deg", C.c_float), ("dy", C.c_int), ("dx", C.c_int),
                ("pce", C.c_double), ("peak", C.c_float), ("cand_idx", C.c_int)]


class prnu_query(C.Structure):
    _fields_ = [("frames", C.c_void_p), ("F", C.c_int), ("H", C.c_int), ("W", C.c_int), ("pitch", C.c_size_t),
                ("fp_handles", C.POINTER(C.c_uint64)), ("P", C.c_int), ("grid", prnu_grid),
                ("windows", C.POINTER(prnu_window)), ("dtype", C.c_int), ("flags", C.c_int)]


class prnu_server_stats(C.Structure):
    _fields_ = [("queries_done", C.c_uint64), ("candidates_done", C.c_uint64), ("server_launches", C.c_uint64),
                ("admitted_bytes_peak", C.c_uint64), ("admitted_bytes_now", C.c_uint64)]


class prnu_tuning(C.Structure):
    _fields_ = [("col_width", C.c_int), ("pairs_per_block", C.c_int), ("wave", C.c_int), ("variant", C.c_int),
                ("persistent", C.c_int), ("streams", C.c_int), ("share_forward", C.c_int)]


class prnu_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_uint64), ("total_ms", C.c_double)]


RESULT_DTYPE = np.dtype([("lam", "<f4"), ("th_deg", "<f4"), ("dy", "<i4"), ("dx", "<i4"), ("pce", "<f8"),
                         ("peak", "<f4"), ("cand_idx", "<i4")])
assert RESULT_DTYPE.itemsize == C.sizeof(prnu_result) == 32

_P = C.c_void_p
_SIGNATURES = {
    "prnu_create": (C.c_int, [C.POINTER(_P), C.c_int, C.c_size_t]),
    "prnu_destroy": (C.c_int, [_P]),
    "prnu_last_error": (C.c_char_p, []),
    "prnu_launch_count": (C.c_uint64, [_P]),
    "prnu_residual": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_size_t, C.c_int, C.c_int, _P, _P, _P]),
    "prnu_fingerprint_term": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_uint64), _P]),
    "prnu_fingerprint_release": (C.c_int, [_P, C.c_uint64]),
    "prnu_fingerprint_estimate": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_size_t, _P, _P]),
    "eis_grid_search": (C.c_int, [_P, _P, C.c_int, _P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_uint64), C.c_int,
                                  C.POINTER(prnu_grid), C.POINTER(prnu_window), _P, _P, _P]),
    "eis_grid_search_naive": (C.c_int, [_P, _P, C.c_int, _P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_uint64),
                                        C.c_int, C.POINTER(prnu_grid), C.POINTER(prnu_window), _P, _P, _P]),
    "prnu_residual_wavelet": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_size_t, C.c_int, C.c_int,
                                        C.c_double, _P, _P, _P]),
    "prnu_fingerprint_resize": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_size_t, C.c_double, C.c_int, C.c_int, _P,
                                          C.c_int, C.c_int, _P]),
    "eis_grid_search_frames": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_size_t, C.c_int,
                                         C.POINTER(C.c_uint64), C.c_int, C.POINTER(prnu_grid),
                                         C.POINTER(prnu_window), _P, _P]),
    "eis_correction": (C.c_int, [_P, _P, C.c_int, _P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_uint64), C.c_int,
                                 _P, _P, C.c_int, C.c_int, _P, _P, _P]),
    "similarity_from_homography": (C.c_int, [_P, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "eis_invert_video": (C.c_int, [_P, _P, C.c_int, _P, C.c_int, C.c_int, C.c_int, C.c_uint64, _P, C.c_int,
                                   C.c_int, C.c_double, _P, C.POINTER(C.c_double), C.POINTER(C.c_int), _P, _P,
                                   _P]),
    "pce_score": (C.c_int, [_P, _P, C.c_uint64, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int),
                            C.POINTER(C.c_int), C.POINTER(C.c_float), _P]),
    "pce_score_noalloc": (C.c_int, [_P, _P, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int),
                                    C.POINTER(C.c_int), C.POINTER(C.c_float), _P]),
    "query_submit": (C.c_int, [_P, C.POINTER(prnu_query), C.POINTER(C.c_uint64)]),
    "query_poll": (C.c_int, [_P, C.c_uint64, _P, C.c_int64]),
    "query_latency": (C.c_int, [_P, C.c_uint64, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "prnu_server_stats_get": (C.c_int, [_P, C.POINTER(prnu_server_stats)]),
    "prnu_server_set_loop": (C.c_int, [_P, C.c_int]),
    "prnu_get_tuning": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(prnu_tuning)]),
    "prnu_set_tuning": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(prnu_tuning)]),
    "prnu_autotune": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_double, C.POINTER(prnu_tuning), _P]),
    "prnu_profile_begin": (C.c_int, [_P]),
    "prnu_profile_end": (C.c_int, [_P, C.POINTER(prnu_kernel_stat), C.c_int, C.POINTER(C.c_int)]),
    "prnu_debug_set": (C.c_int, [_P, C.c_int, C.c_int]),
}
EXPORTED = tuple(_SIGNATURES)

_lib = None


def lib() -> C.CDLL:
    """Load libprnu.so (built by ``build()``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libprnu.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def build(force: bool = False) -> str:
    from .buildlib import build as _build
    return _build(force=force)


def _check(code: int, func: str):
    if code != PRNU_OK:
        raise PrnuError(code, func, lib().prnu_last_error().decode(errors="replace"))


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def make_grid(g) -> prnu_grid:
    return prnu_grid(g.lam0, g.dlam, g.nlam, g.th0_deg, g.dth_deg, g.nth)


def make_windows(windows, F=None):
    """ctypes array of prnu_window from an int array [F, 4] (or None); with F
    given, a count other than F raises PRNU_EINVAL (the library reads F)."""
    if windows is None:
        return None
    w = np.ascontiguousarray(windows, dtype=np.int32).reshape(-1, 4)
    if F is not None and len(w) != F:
        raise PrnuError(PRNU_EINVAL, "windows", f"{len(w)} windows for {F} frames")
    arr = (prnu_window * len(w))()
    for i, (a, b, c, d) in enumerate(w):
        arr[i] = prnu_window(int(a), int(b), int(c), int(d))
    return arr


def similarity_from_homography(Hm):
    """(lambda, theta in degrees) of the similarity nearest to the linear part
    of a 3x3 homography acting on (column, row, 1)."""
    hm = np.ascontiguousarray(np.asarray(Hm, np.float64).reshape(9))
    lam, th = C.c_float(0.0), C.c_float(0.0)
    _check(lib().similarity_from_homography(hm.ctypes.data_as(_P), C.byref(lam), C.byref(th)),
           "similarity_from_homography")
    return lam.value, th.value


def pce_score_noalloc(X, K, stream=None) -> dict:
    """PCE of the aligned pair (X, K) without any device allocation, for callers
    that cannot allocate (see include/prnu.h).  X, K: dense float32 CUDA tensors
    [H, W] on one device, H*W <= 2^20.  The call runs with X's device current,
    on `stream` or that device's current stream."""
    import torch
    if X.dim() != 2 or tuple(K.shape) != tuple(X.shape):
        raise PrnuError(PRNU_EINVAL, "pce_score_noalloc", f"X {tuple(X.shape)} and K {tuple(K.shape)} "
                                                          "must be [H, W] of one size")
    if X.dtype != torch.float32 or K.dtype != torch.float32:
        raise PrnuError(PRNU_EINVAL, "pce_score_noalloc", "X and K must be float32")
    if not (X.is_cuda and K.is_cuda) or X.device != K.device:
        raise PrnuError(PRNU_EINVAL, "pce_score_noalloc", "X and K must be CUDA tensors on one device")
    if not (X.is_contiguous() and K.is_contiguous()):
        raise PrnuError(PRNU_EINVAL, "pce_score_noalloc", "X and K must be contiguous")
    H, W = X.shape
    pce, dy, dx, peak = C.c_double(), C.c_int(), C.c_int(), C.c_float()
    with torch.cuda.device(X.device):
        st = _stream(stream if stream is not None else torch.cuda.current_stream(X.device))
        _check(lib().pce_score_noalloc(_ptr(X), _ptr(K), H, W, C.byref(pce), C.byref(dy), C.byref(dx),
                                       C.byref(peak), st), "pce_score_noalloc")
    return dict(pce=pce.value, dy=dy.value, dx=dx.value, peak=peak.value)


class Context:
    """A libprnu context on one CUDA device (``prnu_create``)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        h = C.c_void_p()
        _check(lib().prnu_create(C.byref(h), device, hbm_budget_bytes), "prnu_create")
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            _check(lib().prnu_destroy(self.h), "prnu_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def prnu_launch_count(self) -> int:
        return int(lib().prnu_launch_count(self.h))

    # --------------------------------------------------------------- hot path
    def prnu_residual(self, frames, out, scale=None, flags=PRNU_WEIGHT_BY_INTENSITY, pitch=0, stream=None):
        """frames: uint8 CUDA tensor [F, H, W]; out: float32/float16/bfloat16 CUDA tensor [F, H, W]."""
        import torch
        F, H, W = frames.shape[-3:]
        dt = {torch.float32: PRNU_F32, torch.float16: PRNU_F16, torch.bfloat16: PRNU_BF16}[out.dtype]
        pitch = pitch or (frames.stride(-2) if frames.dim() >= 2 else W)
        _check(lib().prnu_residual(self.h, _ptr(frames), F, H, W, pitch, flags, dt, _ptr(out), _ptr(scale),
                                   _stream(stream)), "prnu_residual")
        return out

    def prnu_fingerprint_term(self, K, store_dtype=PRNU_F32, stream=None) -> int:
        H, W = K.shape
        h = C.c_uint64()
        _check(lib().prnu_fingerprint_term(self.h, _ptr(K), H, W, store_dtype, C.byref(h), _stream(stream)),
               "prnu_fingerprint_term")
        return int(h.value)

    def prnu_fingerprint_release(self, handle: int):
        _check(lib().prnu_fingerprint_release(self.h, handle), "prnu_fingerprint_release")

    def prnu_fingerprint_estimate(self, frames, out=None, pitch=0, stream=None):
        """Eq. 2 reference fingerprint from frames (CUDA uint8 [L, H, W]); returns
        (or fills) a CUDA float32 tensor [H, W]."""
        import torch
        L, H, W = frames.shape
        if out is None:
            out = torch.empty((H, W), dtype=torch.float32, device=frames.device)
        _check(lib().prnu_fingerprint_estimate(self.h, _ptr(frames), L, H, W, pitch, _ptr(out), _stream(stream)),
               "prnu_fingerprint_estimate")
        return out

    def eis_correction(self, resid, fp_handles, init_lam=None, init_th=None, max_iter=3, th_half1=50, scale=None,
                       stream=None):
        """The iterative correction of Sec. 3.2 for every (frame, fingerprint)
        pair.  resid: CUDA tensor [F, H, W]; init_lam, init_th: array-likes of
        F*P start estimates or None (1 and 0).  Returns (results [F, P] of
        RESULT_DTYPE, iterations run [F, P])."""
        import torch
        F, H, W = resid.shape
        dt = {torch.float32: PRNU_F32, torch.float16: PRNU_F16, torch.bfloat16: PRNU_BF16}[resid.dtype]
        P = len(fp_handles)
        hs = (C.c_uint64 * max(P, 1))(*fp_handles)
        out = np.zeros((F, P), dtype=RESULT_DTYPE)
        its = np.zeros((F, P), dtype=np.int32)
        il = None if init_lam is None else np.ascontiguousarray(np.asarray(init_lam, np.float32).reshape(F * P))
        it_ = None if init_th is None else np.ascontiguousarray(np.asarray(init_th, np.float32).reshape(F * P))
        _check(lib().eis_correction(self.h, _ptr(resid), dt, _ptr(scale), F, H, W, hs, P,
                                    None if il is None else il.ctypes.data_as(_P),
                                    None if it_ is None else it_.ctypes.data_as(_P), max_iter, th_half1,
                                    out.ctypes.data_as(_P), its.ctypes.data_as(_P), _stream(stream)),
               "eis_correction")
        return out, its

    def prnu_residual_wavelet(self, frames, out, sigma0=3.0, flags=PRNU_WEIGHT_BY_INTENSITY, scale=None, pitch=0,
                              stream=None):
        """Residual by Mihcak's wavelet denoiser (Sec. 2.2).  frames: CUDA
        uint8 [F, H, W]; out: CUDA [F, H, W] float32/float16/bfloat16."""
        import torch
        F, H, W = frames.shape
        dt = {torch.float32: PRNU_F32, torch.float16: PRNU_F16, torch.bfloat16: PRNU_BF16}[out.dtype]
        _check(lib().prnu_residual_wavelet(self.h, _ptr(frames), F, H, W, pitch, flags, dt, float(sigma0), _ptr(out),
                                           _ptr(scale), _stream(stream)), "prnu_residual_wavelet")
        return out

    def prnu_fingerprint_resize(self, K, scale, y0, x0, H, W, out=None, stream=None):
        """The fingerprint K (CUDA float tensor [Hin, Win], rows may be
        strided) resized by `scale` and cropped to H x W from (y0, x0)."""
        import torch
        Hin, Win = K.shape
        assert K.dtype == torch.float32 and K.stride(1) == 1
        if out is None:
            out = torch.empty((H, W), dtype=torch.float32, device=K.device)
        _check(lib().prnu_fingerprint_resize(self.h, _ptr(K), Hin, Win, K.stride(0), float(scale), y0, x0, _ptr(out),
                                             H, W, _stream(stream)), "prnu_fingerprint_resize")
        return out

    def eis_grid_search_frames(self, frames, fp_handles, grid, windows=None, flags=PRNU_WEIGHT_BY_INTENSITY,
                               pitch=0, out=None, stream=None):
        """The frame-literal grid search of Sec. 3.2 (warp the frame, extract
        the residual per candidate).  frames: CUDA uint8 tensor [F, H, W] (row
        pitch `pitch` bytes, 0 = W).  Returns results [F, P] of RESULT_DTYPE
        (or fills `out`, a host array or a CUDA byte tensor)."""
        F, H, W = frames.shape[0], frames.shape[1], frames.shape[2]
        P = len(fp_handles)
        hs = (C.c_uint64 * max(P, 1))(*fp_handles)
        g = make_grid(grid)
        win = make_windows(windows, F)
        host = out is None
        if host:
            out = np.zeros((F, P), dtype=RESULT_DTYPE)
        ptr = out.ctypes.data_as(_P) if isinstance(out, np.ndarray) else _ptr(out)
        _check(lib().eis_grid_search_frames(self.h, _ptr(frames), F, H, W, pitch, flags, hs, P, C.byref(g), win,
                                            ptr, _stream(stream)),
               "eis_grid_search_frames")
        return out

    def eis_invert_video(self, resid, fp_handle, homographies=None, max_iter=3, th_half1=50, tau=19.5,
                         scale=None, stream=None):
        """Algorithm 1 with the co-registration supplied, and the decision of
        Sec. 3.2.  resid: CUDA tensor [F, H, W], frame 0 the anchor;
        homographies: array-like [F, 3, 3] (entry 0 unused) or None.  Returns
        dict(gamma [F], mean, decision, best [F] of RESULT_DTYPE, from_reg [F])."""
        import torch
        F, H, W = resid.shape
        dt = {torch.float32: PRNU_F32, torch.float16: PRNU_F16, torch.bfloat16: PRNU_BF16}[resid.dtype]
        hm = None if homographies is None else np.ascontiguousarray(
            np.asarray(homographies, np.float64).reshape(F * 9))
        gamma = np.zeros(F, np.float64)
        best = np.zeros(F, dtype=RESULT_DTYPE)
        from_reg = np.zeros(F, np.int32)
        mean, dec = C.c_double(0.0), C.c_int(0)
        _check(lib().eis_invert_video(self.h, _ptr(resid), dt, _ptr(scale), F, H, W, fp_handle,
                                      None if hm is None else hm.ctypes.data_as(_P), max_iter, th_half1, tau,
                                      gamma.ctypes.data_as(_P), C.byref(mean), C.byref(dec),
                                      best.ctypes.data_as(_P), from_reg.ctypes.data_as(_P), _stream(stream)),
               "eis_invert_video")
        return dict(gamma=gamma, mean=mean.value, decision=bool(dec.value), best=best,
                    from_reg=from_reg.astype(bool))

    def eis_grid_search(self, resid, fp_handles, grid, windows=None, scale=None, out=None, all_pce=None,
                        stream=None, naive=False):
        """resid: CUDA tensor [F, H, W] (float32/float16/bfloat16).  Returns a numpy
        structured array [F, P] of results (RESULT_DTYPE) when ``out`` is None,
        else fills the CUDA uint8/float tensor ``out`` (F*P*32 bytes)."""
        import torch
        F, H, W = resid.shape
        dt = {torch.float32: PRNU_F32, torch.float16: PRNU_F16, torch.bfloat16: PRNU_BF16}[resid.dtype]
        P = len(fp_handles)
        hs = (C.c_uint64 * max(P, 1))(*fp_handles)
        g = make_grid(grid)
        w = make_windows(windows, F)
        host = out is None
        if host:
            res = np.zeros((F, P), dtype=RESULT_DTYPE)
            optr = C.c_void_p(res.ctypes.data)
        else:
            res = out
            optr = _ptr(out)
        fn = lib().eis_grid_search_naive if naive else lib().eis_grid_search
        _check(fn(self.h, _ptr(resid), dt, _ptr(scale), F, H, W, hs, P, C.byref(g), w, optr, _ptr(all_pce),
                  _stream(stream)), "eis_grid_search_naive" if naive else "eis_grid_search")
        return res

    def pce_score(self, X, handle: int, stream=None):
        H, W = X.shape
        pce, dy, dx, peak = C.c_double(), C.c_int(), C.c_int(), C.c_float()
        _check(lib().pce_score(self.h, _ptr(X), handle, H, W, C.byref(pce), C.byref(dy), C.byref(dx),
                               C.byref(peak), _stream(stream)), "pce_score")
        return dict(pce=pce.value, dy=dy.value, dx=dx.value, peak=peak.value)

    # --------------------------------------------------------------- serving
    def query_submit(self, frames, fp_handles, grid, windows=None, dtype=PRNU_F16,
                     flags=PRNU_WEIGHT_BY_INTENSITY | PRNU_NORMALISE) -> int:
        """frames: uint8 tensor [F, H, W] on the device or in (pinned) host memory;
        it must stay alive until query_poll returns the results."""
        F, H, W = frames.shape
        P = len(fp_handles)
        hs = (C.c_uint64 * max(P, 1))(*fp_handles)
        w = make_windows(windows, F)
        q = prnu_query(C.c_void_p(frames.data_ptr()), F, H, W, frames.stride(1), hs, P, make_grid(grid),
                       w, dtype, flags)
        qid = C.c_uint64()
        _check(lib().query_submit(self.h, C.byref(q), C.byref(qid)), "query_submit")
        return int(qid.value)

    def query_poll(self, qid: int, F: int, P: int, timeout_us: int = -1):
        """Returns the [F, P] results, or None while the query is not done."""
        res = np.zeros((F, P), dtype=RESULT_DTYPE)
        code = lib().query_poll(self.h, qid, C.c_void_p(res.ctypes.data), timeout_us)
        if code in (PRNU_EAGAIN, PRNU_ETIMEOUT):
            return None
        _check(code, "query_poll")
        return res

    def query_latency(self, qid: int) -> dict:
        qm, tm = C.c_double(), C.c_double()
        _check(lib().query_latency(self.h, qid, C.byref(qm), C.byref(tm)), "query_latency")
        return dict(queued_ms=qm.value, total_ms=tm.value)

    def prnu_server_set_loop(self, mode):
        """PRNU_LOOP_HOST or PRNU_LOOP_DEVICE; before the first query_submit."""
        _check(lib().prnu_server_set_loop(self.h, int(mode)), "prnu_server_set_loop")

    def prnu_server_stats_get(self) -> dict:
        s = prnu_server_stats()
        _check(lib().prnu_server_stats_get(self.h, C.byref(s)), "prnu_server_stats_get")
        return {k: int(getattr(s, k)) for k, _ in s._fields_}

    # --------------------------------------------------------------- profiling
    def prnu_profile_begin(self):
        _check(lib().prnu_profile_begin(self.h), "prnu_profile_begin")

    def prnu_profile_end(self) -> dict:
        arr = (prnu_kernel_stat * 32)()
        n = C.c_int()
        _check(lib().prnu_profile_end(self.h, arr, 32, C.byref(n)), "prnu_profile_end")
        return {arr[i].name.decode(): dict(launches=int(arr[i].launches), total_ms=float(arr[i].total_ms))
                for i in range(min(n.value, 32))}

    # --------------------------------------------------------------- tuning
    def prnu_get_tuning(self, H, W) -> dict:
        t = prnu_tuning()
        _check(lib().prnu_get_tuning(self.h, H, W, C.byref(t)), "prnu_get_tuning")
        return dict(col_width=t.col_width, pairs_per_block=t.pairs_per_block, wave=t.wave, variant=t.variant,
                    persistent=t.persistent, streams=t.streams, share_forward=t.share_forward)

    def prnu_debug_set(self, key, value):
        _check(lib().prnu_debug_set(self.h, key, value), "prnu_debug_set")

    def prnu_set_tuning(self, H, W, col_width, pairs_per_block, wave, variant=0, persistent=0, streams=1,
                        share_forward=1):
        t = prnu_tuning(col_width, pairs_per_block, wave, variant, persistent, streams, share_forward)
        _check(lib().prnu_set_tuning(self.h, H, W, C.byref(t)), "prnu_set_tuning")

    def prnu_autotune(self, H, W, dtype=PRNU_F32, budget_ms=2000.0, stream=None) -> dict:
        t = prnu_tuning()
        _check(lib().prnu_autotune(self.h, H, W, dtype, budget_ms, C.byref(t), _stream(stream)), "prnu_autotune")
        return dict(col_width=t.col_width, pairs_per_block=t.pairs_per_block, wave=t.wave, variant=t.variant,
                    persistent=t.persistent, streams=t.streams, share_forward=t.share_forward)
