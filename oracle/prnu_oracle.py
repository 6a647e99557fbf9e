"""Plain FP64 CPU oracle of the EIS-inversion grid search.  TEST INFRASTRUCTURE.

What it computes (arXiv 2207.14507):

* noise residual W(I) = I - F(I)                                   (Sec. 2.2)
  with F a 3x3 local Wiener filter (the workloads replace the wavelet
  denoiser of Sec. 2.2 by a 3x3 Wiener filter), weighted by the frame
  intensity, R = I * W(I), the fingerprint-matching term of Eq. 2/3;
* the wavelet-domain residual of Mihcak's denoiser (the paper's
  denoiser, Sec. 2.2): 4-level orthonormal 8-tap Daubechies
  transform, local-variance Wiener shrinkage of the detail bands     (Sec. 2.2)
* fingerprint term K0 = K - mean(K)                                 (Eq. 1, 3)
* reference fingerprint from L frames,
  K = (sum_l I_l W(I_l)) / (sum_l I_l^2), pixel-wise                (Eq. 2)
* the fingerprint down-scaled and cropped to the video geometry     (Sec. 3)
* inverse similarity warp of R, bilinear, zero outside the frame    (Eq. 4, Sec. 3.2)
* circular cross-correlation over all shifts, C(d) = sum_x X(x) K0(x + d)
* PCE with an 11x11 cyclic exclusion around the signed peak         (Eq. 3)
* exhaustive search over the (lambda, theta) grid, arg-max PCE      (Sec. 3.2, Eq. 8)
* the frame-literal variant: per candidate, warp the frame and take
  the residual of the warped frame                                  (Sec. 3.2)
* the iterative breadth-first correction: progressively narrower
  (lambda, theta) neighbourhoods of the previous estimate          (Sec. 3.2, Eq. 8)
* the EIS inversion of a video segment with the co-registration
  supplied, the PCE vector gamma and its thresholded mean          (Algorithm 1, Sec. 3.2)

Everything is float64 NumPy, written as the plain definition; the only library
primitives are numpy's FFTs (for the correlation) and array arithmetic.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this module.  It shares no code with the CUDA path, and the CUDA path
never calls it.

Parity pins (see tests/test_oracle_pins.py): brute-force direct correlation on
32x32 and 30x40; closed-form warps (identity, 90-degree rotation, 2x zoom);
PCE of a delta-plus-constant surface and of a brute-force masked surface;
invariance of the PCE to global gain and to a common cyclic shift; Wiener
residual against scipy's reference filter in the interior and against
scipy.ndimage's replicate-padded moments; planted-transform recovery.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "EXCLUSION", "local_moments_3x3", "wiener_residual", "prnu_residual",
    "DB8", "dwt2_level", "idwt2_level", "dwt2", "idwt2", "mihcak_shrink", "wavelet_residual", "prnu_residual_wavelet",
    "fingerprint_term", "grid_lambda", "grid_theta", "warp_matrix", "inverse_warp",
    "xcorr", "pce", "score", "grid_search", "candidate_list", "ncc_peak",
    "literal_residual", "score_literal", "grid_search_literal",
    "correction_nodes", "correction", "fingerprint_estimate", "resize_weights", "fingerprint_resize", "similarity_from_homography", "invert_video", "TAU",
]

# Eq. 3: the exclusion neighbourhood D around the correlation peak is 11 x 11, cyclic.
EXCLUSION = 11


# ----------------------------------------------------------------------------- residual (Sec. 2.2)

def local_moments_3x3(I: np.ndarray):
    """3x3 local mean and population variance, borders replicated."""
    I = np.asarray(I, dtype=np.float64)
    H, W = I.shape
    P = np.pad(I, 1, mode="edge")
    s1 = np.zeros((H, W))
    s2 = np.zeros((H, W))
    for dy in range(3):
        for dx in range(3):
            v = P[dy:dy + H, dx:dx + W]
            s1 += v
            s2 += v * v
    mu = s1 / 9.0
    var = s2 / 9.0 - mu * mu
    return mu, var


def wiener_residual(I: np.ndarray):
    """W(I) = I - Wiener3x3(I) with the noise power nu^2 = mean of the local variances.

    Wiener3x3(I) = mu + (I - mu) * max(var - nu^2, 0) / max(var, nu^2); where both
    var and nu^2 are zero the window is constant, I == mu and W = 0.
    Returns (W, nu^2).
    """
    I = np.asarray(I, dtype=np.float64)
    mu, var = local_moments_3x3(I)
    nu2 = float(var.mean())
    den = np.maximum(var, nu2)
    safe = np.where(den > 0, den, 1.0)
    gain = np.where(den > 0, np.maximum(var - nu2, 0.0) / safe, 1.0)
    wien = mu + (I - mu) * gain
    return I - wien, nu2


def prnu_residual(frame: np.ndarray, weight_by_intensity: bool = True, normalise: bool = False):
    """Residual fed to the matcher: R = I * W(I) (default) or W(I).

    With ``normalise`` R is multiplied by s = 1 / RMS(R) (s = 1 when R == 0).
    Returns (R, s).
    """
    I = np.asarray(frame, dtype=np.float64)
    Wr, _ = wiener_residual(I)
    R = I * Wr if weight_by_intensity else Wr
    s = 1.0
    if normalise:
        ms = float(np.mean(R * R))
        s = 1.0 / np.sqrt(ms) if ms > 0 else 1.0
        R = R * s
    return R, s


# ----------------------------------------------------------------------------- Mihcak denoiser (Sec. 2.2)

# Daubechies' orthonormal scaling filter with 4 vanishing moments (8 taps),
# normalised to sum sqrt(2).  The wavelet filter is g[k] = (-1)^k h[7 - k].
DB8 = np.array([0.2303778133088964, 0.7148465705529154, 0.6308807679298587, -0.0279837694168599,
                -0.1870348117190931, 0.0308413818355607, 0.0328830116668852, -0.0105974017850690])
WAVELET_LEVELS = 4


def _wavelet_filter(h):
    return np.array([(-1) ** k * h[len(h) - 1 - k] for k in range(len(h))])


def _analysis_1d(x, axis):
    """Periodic analysis along `axis`: a[n] = sum_k h[k] x[2n + k], d[n] = sum_k g[k] x[2n + k]."""
    g = _wavelet_filter(DB8)
    a = np.zeros_like(np.take(x, np.arange(0, x.shape[axis], 2), axis=axis))
    d = np.zeros_like(a)
    for k in range(len(DB8)):
        xs = np.take(np.roll(x, -k, axis=axis), np.arange(0, x.shape[axis], 2), axis=axis)
        a += DB8[k] * xs
        d += g[k] * xs
    return a, d


def _synthesis_1d(a, d, axis):
    """The transpose of _analysis_1d (its inverse, the filters being orthonormal)."""
    g = _wavelet_filter(DB8)
    shape = list(a.shape)
    shape[axis] *= 2
    x = np.zeros(shape)
    up_a, up_d = np.zeros(shape), np.zeros(shape)
    idx = [slice(None)] * len(shape)
    idx[axis] = slice(0, None, 2)
    up_a[tuple(idx)] = a
    up_d[tuple(idx)] = d
    for k in range(len(DB8)):
        x += DB8[k] * np.roll(up_a, k, axis=axis) + g[k] * np.roll(up_d, k, axis=axis)
    return x


def dwt2_level(X):
    """One level of the separable 2-D transform (rows, then columns):
    returns (LL, (LH, HL, HH)) with L/H the row filter first."""
    L, Hh = _analysis_1d(X, axis=1)
    LL, LH = _analysis_1d(L, axis=0)
    HL, HH = _analysis_1d(Hh, axis=0)
    return LL, (LH, HL, HH)


def idwt2_level(LL, bands):
    LH, HL, HH = bands
    L = _synthesis_1d(LL, LH, axis=0)
    Hh = _synthesis_1d(HL, HH, axis=0)
    return _synthesis_1d(L, Hh, axis=1)


def dwt2(X, levels: int = WAVELET_LEVELS):
    """Multi-level transform of the approximation band: (LL, [bands of level 1, 2, ...])."""
    details = []
    A = np.asarray(X, dtype=np.float64)
    for _ in range(levels):
        A, b = dwt2_level(A)
        details.append(b)
    return A, details


def idwt2(A, details):
    for b in reversed(details):
        A = idwt2_level(A, b)
    return A


def mihcak_shrink(c, sigma0: float):
    """The noise part of one detail band: c sigma0^2 / (s2 + sigma0^2), where
    s2 = min over W in {3, 5, 7, 9} of max(0, mean of c^2 over the W x W window
    - sigma0^2), the window mean over W^2 positions with zeros outside the
    band.  Where s2 + sigma0^2 = 0 the noise part is 0."""
    c = np.asarray(c, dtype=np.float64)
    c2 = c * c
    s2 = None
    for Wn in (3, 5, 7, 9):
        r = Wn // 2
        P = np.pad(c2, r)
        acc = np.zeros_like(c2)
        for dy in range(Wn):
            for dx in range(Wn):
                acc += P[dy:dy + c.shape[0], dx:dx + c.shape[1]]
        v = np.maximum(acc / (Wn * Wn) - sigma0 ** 2, 0.0)
        s2 = v if s2 is None else np.minimum(s2, v)
    den = s2 + sigma0 ** 2
    return np.where(den > 0, c * sigma0 ** 2 / np.where(den > 0, den, 1.0), 0.0)


def wavelet_residual(I, sigma0: float = 3.0, levels: int = WAVELET_LEVELS):
    """W(I) = I - F(I) with F Mihcak's denoiser: the frame mirrored at its
    bottom and right edges up to multiples of 2^levels, the detail bands of
    every level replaced by their noise parts (mihcak_shrink), the
    approximation band by 0, the inverse transform cropped back to the frame
    (the transform is linear, so this is the frame minus its denoised version)."""
    I = np.asarray(I, dtype=np.float64)
    H, W = I.shape
    m = 2 ** levels
    Hp, Wp = -(-H // m) * m, -(-W // m) * m
    P = np.pad(I, ((0, Hp - H), (0, Wp - W)), mode="symmetric")
    A, det = dwt2(P, levels)
    det = [tuple(mihcak_shrink(b, sigma0) for b in lv) for lv in det]
    return idwt2(np.zeros_like(A), det)[:H, :W]


def prnu_residual_wavelet(frame, sigma0: float = 3.0, weight_by_intensity: bool = True):
    """R = I * W(I) (or W(I)) with the wavelet residual."""
    I = np.asarray(frame, dtype=np.float64)
    Wr = wavelet_residual(I, sigma0)
    return I * Wr if weight_by_intensity else Wr


def fingerprint_term(K: np.ndarray) -> np.ndarray:
    """K0 = K - mean(K): the mean-removed fingerprint of the NCC (Eq. 1)."""
    K = np.asarray(K, dtype=np.float64)
    return K - K.mean()


# ----------------------------------------------------------------------------- candidates (Sec. 3.2)

def _f32(x) -> float:
    return float(np.float32(x))


def grid_lambda(lam0: float, dlam: float, i: int) -> float:
    """Scale node i: lam0 + i*dlam from float32 descriptor fields, evaluated in
    float64 and rounded to float32 (the value both sides search)."""
    return _f32(_f32(lam0) + i * _f32(dlam))


def grid_theta(th0: float, dth: float, j: int) -> float:
    return _f32(_f32(th0) + j * _f32(dth))


def candidate_list(grid, window=None):
    """(index, lambda, theta_deg) of every candidate, lambda-major, index = i*nth + j.

    ``window`` = (lam_lo, lam_hi, th_lo, th_hi), inclusive; None = full grid.
    """
    lo_i, hi_i, lo_j, hi_j = (0, grid.nlam - 1, 0, grid.nth - 1) if window is None else window
    out = []
    for i in range(lo_i, hi_i + 1):
        for j in range(lo_j, hi_j + 1):
            out.append((i * grid.nth + j, grid_lambda(grid.lam0, grid.dlam, i),
                        grid_theta(grid.th0_deg, grid.dth_deg, j)))
    return out


# ----------------------------------------------------------------------------- warp (Eq. 4)

def warp_matrix(lam: float, theta_deg: float) -> np.ndarray:
    """A = Rot(-theta) / lambda, so that q = c + A (p - c) maps a corrected pixel p
    to the stabilised frame.  Eq. 4 restricted as in Sec. 3.2: t11 = t22 = scale,
    t12 = -t21 = rotation, no projective terms; the translation is left to the
    correlation peak.  Rot acts on (x = column, y = row)."""
    th = np.deg2rad(theta_deg)
    c, s = np.cos(th), np.sin(th)
    return np.array([[c, s], [-s, c]]) / lam


def inverse_warp(R: np.ndarray, lam: float, theta_deg: float) -> np.ndarray:
    """X(p) = bilinear(R, q), q = c + A (p - c), c = ((W-1)/2, (H-1)/2).

    Each of the four bilinear taps that falls outside the frame contributes 0.
    """
    R = np.asarray(R, dtype=np.float64)
    H, W = R.shape
    cy, cx = (H - 1) / 2.0, (W - 1) / 2.0
    A = warp_matrix(lam, theta_deg)
    yy, xx = np.meshgrid(np.arange(H) - cy, np.arange(W) - cx, indexing="ij")
    qx = cx + A[0, 0] * xx + A[0, 1] * yy
    qy = cy + A[1, 0] * xx + A[1, 1] * yy
    x0 = np.floor(qx)
    y0 = np.floor(qy)
    fx = qx - x0
    fy = qy - y0
    x0 = x0.astype(np.int64)
    y0 = y0.astype(np.int64)
    X = np.zeros((H, W))
    for oy, wy in ((0, 1.0 - fy), (1, fy)):
        for ox, wx in ((0, 1.0 - fx), (1, fx)):
            yi = y0 + oy
            xi = x0 + ox
            ok = (yi >= 0) & (yi < H) & (xi >= 0) & (xi < W)
            vals = np.zeros((H, W))
            vals[ok] = R[yi[ok], xi[ok]]
            X += wy * wx * vals
    return X


# ----------------------------------------------------------------------------- correlation and PCE (Eq. 1, 3)

def xcorr(X: np.ndarray, K0: np.ndarray, K0_spectrum: np.ndarray | None = None) -> np.ndarray:
    """Circular cross-correlation over all shifts, C(d) = sum_x X(x) K0((x + d) mod (H, W)).

    The NCC normalisation of Eq. 1 is a constant over d and cancels in the PCE,
    so it is left out here (see ``ncc_peak``).
    """
    H, W = X.shape
    FK = np.fft.rfft2(K0) if K0_spectrum is None else K0_spectrum
    return np.fft.irfft2(np.conj(np.fft.rfft2(X)) * FK, s=(H, W))


def pce(C: np.ndarray, exclusion: int = EXCLUSION):
    """Peak-to-correlation energy, Eq. 3.

    The peak is the signed maximum of C (first in row-major order on ties); the
    energy is the mean of C^2 over all shifts outside the cyclic
    exclusion x exclusion window centred on the peak.  PCE = sgn(C*) C*^2 / E,
    with E == 0 giving 0 for a zero peak and +-inf otherwise.
    Returns dict(pce, dy, dx, peak, py, px) with the shift in [-H/2, H/2) x [-W/2, W/2).
    """
    C = np.asarray(C, dtype=np.float64)
    H, W = C.shape
    flat = int(np.argmax(C))
    py, px = divmod(flat, W)
    peak = float(C[py, px])
    h = exclusion // 2
    mask = np.ones((H, W), dtype=bool)
    mask[np.ix_((py + np.arange(-h, h + 1)) % H, (px + np.arange(-h, h + 1)) % W)] = False
    E = float(np.mean(C[mask] ** 2))
    if E > 0:
        val = float(np.sign(peak) * peak * peak / E)
    else:
        val = 0.0 if peak == 0 else float(np.sign(peak) * np.inf)
    dy = py if py < H / 2 else py - H
    dx = px if px < W / 2 else px - W
    return dict(pce=val, dy=int(dy), dx=int(dx), peak=peak, py=int(py), px=int(px), energy=E)


def ncc_peak(X: np.ndarray, K0: np.ndarray, peak: float) -> float:
    """rho at the peak (Eq. 1): the correlation divided by ||X - mean X|| ||K0 - mean K0||."""
    Xc = X - X.mean()
    Kc = K0 - K0.mean()
    den = np.linalg.norm(Xc) * np.linalg.norm(Kc)
    return float(peak / den) if den > 0 else 0.0


def score(R: np.ndarray, K0: np.ndarray, lam: float, theta_deg: float, K0_spectrum=None):
    """PCE of one candidate: warp, correlate, Eq. 3."""
    X = inverse_warp(R, lam, theta_deg)
    return pce(xcorr(X, K0, K0_spectrum))


# ----------------------------------------------------------------------------- frame-literal variant (Sec. 3.2)

def literal_residual(frame: np.ndarray, lam: float, theta_deg: float, weight_by_intensity: bool = True):
    """Sec. 3.2 as printed: warp the frame I by the candidate, X = inverse_warp(I),
    then take the residual of X, R = X * W(X) (or W(X)), with W the same 3x3
    Wiener residual as for frames (borders replicated, noise power the mean
    local variance of X)."""
    X = inverse_warp(np.asarray(frame, dtype=np.float64), lam, theta_deg)
    Wx, _ = wiener_residual(X)
    return X * Wx if weight_by_intensity else Wx


def score_literal(frame, K0, lam: float, theta_deg: float, weight_by_intensity: bool = True, K0_spectrum=None):
    """PCE of one candidate of the frame-literal variant: the residual of the
    warped frame, correlated with K0 as it stands (no further warp), Eq. 3."""
    R = literal_residual(frame, lam, theta_deg, weight_by_intensity)
    return pce(xcorr(R, K0, K0_spectrum))


def grid_search_literal(frames, fingerprints, grid, windows=None, weight_by_intensity: bool = True):
    """grid_search with score_literal: best[f][p] and all_pce as grid_search."""
    F, P = len(frames), len(fingerprints)
    all_pce = np.full((F, P, grid.nlam * grid.nth), np.nan)
    spectra = [np.fft.rfft2(K0) for K0 in fingerprints]
    best = []
    for f in range(F):
        win = None if windows is None else tuple(int(v) for v in windows[f])
        cands = candidate_list(grid, win)
        Rs = [(idx, lam, th, literal_residual(frames[f], lam, th, weight_by_intensity)) for idx, lam, th in cands]
        row = []
        for p in range(P):
            b = None
            for idx, lam, th, R in Rs:
                r = pce(xcorr(R, fingerprints[p], spectra[p]))
                all_pce[f, p, idx] = r["pce"]
                if b is None or r["pce"] > b["pce"]:
                    b = dict(r, lam=lam, th_deg=th, cand=idx)
            row.append(b)
        best.append(row)
    return best, all_pce


# ----------------------------------------------------------------------------- search (Sec. 3.2)

def grid_search(residuals, fingerprints, grid, windows=None, on_candidate=None):
    """Exhaustive search of every frame against every fingerprint.

    residuals: [F, H, W] (R from ``prnu_residual``); fingerprints: list of K0 (mean removed)
    grid: object with lam0, dlam, nlam, th0_deg, dth_deg, nth
    windows: None or int [F, 4] inclusive (lam_lo, lam_hi, th_lo, th_hi) per frame.
    Returns (best, all_pce): best[f][p] = dict(pce, dy, dx, peak, lam, th_deg, cand);
    all_pce: float64 [F, P, nlam*nth], NaN where a candidate was not evaluated.
    Ties in PCE go to the lowest candidate index (lambda-major).
    """
    F = len(residuals)
    P = len(fingerprints)
    all_pce = np.full((F, P, grid.nlam * grid.nth), np.nan)
    spectra = [np.fft.rfft2(K0) for K0 in fingerprints]
    best = []
    for f in range(F):
        row = []
        win = None if windows is None else tuple(int(v) for v in windows[f])
        cands = candidate_list(grid, win)
        for p in range(P):
            b = None
            for idx, lam, th in cands:
                r = score(residuals[f], fingerprints[p], lam, th, spectra[p])
                all_pce[f, p, idx] = r["pce"]
                if on_candidate is not None:
                    on_candidate(f, p, idx, r)
                if b is None or r["pce"] > b["pce"]:
                    b = dict(r, lam=lam, th_deg=th, cand=idx)
            row.append(b)
        best.append(row)
    return best, all_pce


# ----------------------------------------------------------------------------- correction (Sec. 3.2, Eq. 8)

# Reading of Eq. 8, whose printed step sizes (0.01^-n, 0.1^-n) would widen the
# neighbourhoods: iteration n searches lambda(n-1) + a * 0.01 * 10^-(n-1) and
# theta(n-1) + b * 0.1 * 10^-(n-1) degrees for a, b in -5..5, except that the
# first iteration takes theta on the denser grid of the text, b in -50..50
# (-5..5 degrees in steps of 0.1 around the start).  Node values are float32,
# rounded once from the float64 sum of the float32 centre and a * float32(step).
CORR_HALF = 5
CORR_HALF_TH1 = 50


def _corr_step(n: int):
    return _f32(0.01 * 10.0 ** -(n - 1)), _f32(0.1 * 10.0 ** -(n - 1))


def correction_nodes(lam_c: float, th_c: float, n: int, th_half1: int = CORR_HALF_TH1):
    """Scale and angle nodes of iteration n (1-based) around the centre
    (lam_c, th_c): returns (lams, ths), float values of float32 nodes."""
    sl, st = _corr_step(n)
    hb = th_half1 if n == 1 else CORR_HALF
    lams = [_f32(float(np.float32(lam_c)) + a * sl) for a in range(-CORR_HALF, CORR_HALF + 1)]
    ths = [_f32(float(np.float32(th_c)) + b * st) for b in range(-hb, hb + 1)]
    return lams, ths


def correction(R: np.ndarray, K0: np.ndarray, lam0: float = 1.0, th0: float = 0.0, max_iter: int = 3,
               th_half1: int = CORR_HALF_TH1, K0_spectrum=None, score_nodes=None):
    """The correction operator of Sec. 3.2 for one frame residual R and one
    fingerprint term K0: at each iteration an exhaustive search over the
    iteration's nodes (ties to the lowest index, scale-major); stop when the
    best node is the previous estimate (the centre) or after max_iter
    iterations.  Returns (best, iters, path): best = dict of the highest PCE
    seen over all iterations (earliest on ties) with lam, th_deg, cand (index in
    its iteration's node grid), iter (1-based); path = the estimate after each
    iteration.  ``score_nodes`` (optional) scores a list of (lam, th) nodes of R
    and K0 in order, e.g. a ``parallel.ScorePool`` of the same R and K0; by
    default each node is scored here, one after the other."""
    if K0_spectrum is None:
        K0_spectrum = np.fft.rfft2(K0)
    lam_c, th_c = _f32(lam0), _f32(th0)
    best, path = None, []
    n = 0
    for n in range(1, max_iter + 1):
        lams, ths = correction_nodes(lam_c, th_c, n, th_half1)
        nb = len(ths)
        nodes = [(lam, th) for lam in lams for th in ths]
        if score_nodes is None:
            scores = [score(R, K0, lam, th, K0_spectrum) for lam, th in nodes]
        else:
            scores = list(score_nodes(nodes))
        it_best = None
        for c, ((lam, th), r) in enumerate(zip(nodes, scores)):
            if it_best is None or r["pce"] > it_best["pce"]:
                it_best = dict(r, lam=lam, th_deg=th, cand=c, iter=n)
        if best is None or it_best["pce"] > best["pce"]:
            best = it_best
        path.append((it_best["lam"], it_best["th_deg"]))
        centre = CORR_HALF * nb + (nb - 1) // 2
        if it_best["cand"] == centre:
            break
        lam_c, th_c = it_best["lam"], it_best["th_deg"]
    return best, n, path


# ----------------------------------------------------------------------------- fingerprint estimation (Eq. 2)

def fingerprint_estimate(frames) -> np.ndarray:
    """Eq. 2: the reference fingerprint of a device from L of its frames,
    K = (sum_l I_l * W(I_l)) / (sum_l I_l * I_l), every operation pixel-wise,
    with W the residual of ``prnu_residual``; 0 where the denominator is 0."""
    num = None
    den = None
    for frame in frames:
        I = np.asarray(frame, dtype=np.float64)
        R = prnu_residual(I, weight_by_intensity=True)[0]          # I * W(I)
        num = R if num is None else num + R
        den = I * I if den is None else den + I * I
    out = np.zeros_like(num)
    np.divide(num, den, out=out, where=den > 0)
    return out


# ----------------------------------------------------------------------------- fingerprint geometry (Sec. 3)

def resize_weights(n_in: int, scale: float, first: int, n_out: int) -> np.ndarray:
    """[n_out, n_in] weights of output samples first .. first + n_out - 1 of a
    1-D signal of n_in samples resized by `scale`: output sample o sits at
    input position u = (o + 0.5) / scale - 0.5 (pixel centres aligned); its
    weights follow the tent max(0, 1 - |j - u| * a), a = min(scale, 1) (the
    tent widened by 1/scale when shrinking, so that every input sample
    contributes), normalised to sum 1; input indices beyond the ends take the
    end sample (replicated border)."""
    a = min(float(scale), 1.0)
    Wm = np.zeros((n_out, n_in))
    for r in range(n_out):
        u = (first + r + 0.5) / scale - 0.5
        lo, hi = int(np.floor(u - 1.0 / a)), int(np.ceil(u + 1.0 / a))
        w = {}
        for j in range(lo, hi + 1):
            t = max(0.0, 1.0 - abs(j - u) * a)
            if t > 0.0:
                jj = min(max(j, 0), n_in - 1)
                w[jj] = w.get(jj, 0.0) + t
        tot = sum(w.values())
        for jj, t in w.items():
            Wm[r, jj] = t / tot
    return Wm


def fingerprint_resize(K: np.ndarray, scale: float, y0: int, x0: int, H: int, W: int) -> np.ndarray:
    """The fingerprint resized by `scale` (separable, resize_weights along
    rows and columns) and cropped to H x W from (y0, x0) of the resized grid:
    the image fingerprint brought to a video's geometry."""
    K = np.asarray(K, dtype=np.float64)
    Wy = resize_weights(K.shape[0], scale, y0, H)
    Wx = resize_weights(K.shape[1], scale, x0, W)
    return Wy @ K @ Wx.T


# ----------------------------------------------------------------------------- EIS inversion (Algorithm 1)

# Decision threshold on the mean of gamma: the paper's tau for a false-positive
# rate of about 0.05 (Table 1).
TAU = 19.5


def similarity_from_homography(Hm):
    """(lam, th_deg) of the similarity lam * Rot(th) nearest (Frobenius) to the
    linear part of the homography Hm (3x3, acting on (column, row, 1)), via the
    polar decomposition M = R S: R = U V^T is the closest rotation and lam the
    mean singular value.  Sec. 3.2 keeps only scale and rotation of the
    initialising transform.  This is the forward map of the correction node
    (lam, th), i.e. the inverse of warp_matrix(lam, th).  det(M) > 0 only."""
    Hm = np.asarray(Hm, dtype=np.float64).reshape(3, 3)
    M = Hm[:2, :2] / Hm[2, 2]
    if not np.linalg.det(M) > 0:
        raise ValueError("linear part is not orientation preserving")
    U, S, Vt = np.linalg.svd(M)
    R = U @ Vt
    return float(S.mean()), float(np.rad2deg(np.arctan2(R[1, 0], R[0, 0])))


def invert_video(residuals, K0, homographies=None, max_iter: int = 3, th_half1: int = CORR_HALF_TH1,
                 tau: float = TAU):
    """Algorithm 1 with the co-registration supplied by the caller.

    residuals: [F] frame residuals, frame 0 the anchor; K0: fingerprint term.
    homographies: None, or [F] 3x3 homographies H_v that co-register frame v
    with the corrected previous frame (entry 0 unused).  The anchor is
    corrected from (1, 0).  Frame v >= 1 is corrected from the similarity of
    H_v (rounded to float32) if its PCE warped by it exceeds its PCE unwarped,
    else from (1, 0).  gamma[v] is the best PCE of the correction; the
    decision is mean(gamma) > tau.
    Returns dict(gamma, mean, decision, best (per frame), from_reg (per frame))."""
    FK = np.fft.rfft2(K0)
    gamma, bests, from_reg = [], [], []
    for v, R in enumerate(residuals):
        lam0, th0, use = 1.0, 0.0, False
        if v > 0 and homographies is not None:
            rl, rt = similarity_from_homography(homographies[v])
            rl, rt = _f32(rl), _f32(rt)
            if score(R, K0, rl, rt, FK)["pce"] > score(R, K0, 1.0, 0.0, FK)["pce"]:
                lam0, th0, use = rl, rt, True
        best, _, _ = correction(R, K0, lam0, th0, max_iter, th_half1, FK)
        gamma.append(best["pce"])
        bests.append(best)
        from_reg.append(use)
    m = float(np.mean(gamma))
    return dict(gamma=gamma, mean=m, decision=m > tau, best=bests, from_reg=from_reg)
