"""Seeded generators for the five synthetic workloads.

Recipe (stand-in for stabilised VISION videos, which are not available):

* fingerprint K: i.i.d. N(0, 0.02^2) per pixel (float32);
* content: an N(0,1) field blurred by a circular Gaussian (sigma = 8 px),
  min-max scaled to [16, 240];
* sensor frame O = content * (1 + K) + N(0, 2^2);
* electronic stabilisation S(q) = O(T(q)), T(q) = lam * Rot(theta) (q - c) + c + s,
  c = ((W-1)/2, (H-1)/2), sampled bilinearly with edge replication (so that
  stabilised frames carry no black borders);
* quantisation: round half to even, clip to [0, 255], uint8.

Seeds: PCG64 seeded with 2207_14507 + 100 * config + stream (stream 0 = K,
1 = content, 2 = sensor noise, 3 = transforms / windows, 4 = arrivals), with a
spawn key for independent variants (e.g. a second, non-matching fingerprint).

The warp used here is the *forward* stabilisation model applied through
``scipy.ndimage.map_coordinates``; it is data synthesis, not the detector's
inverse warp, and neither the oracle nor the CUDA path uses it.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy import ndimage

__all__ = [
    "BASE_SEED", "Grid", "GRID_C1", "GRID_FULL", "Workload", "rng_for",
    "fingerprint_field", "content_field", "sensor_frame", "stabilise",
    "quantise", "make_frames", "make_workload", "snap_windows",
    "ServingQuery", "make_query_stream",
]

BASE_SEED = 2207_14507
STREAM_K, STREAM_CONTENT, STREAM_NOISE, STREAM_TRANSFORM, STREAM_ARRIVALS = range(5)


def rng_for(config: int, stream: int, variant: int = 0) -> np.random.Generator:
    seed = BASE_SEED + 100 * config + stream
    if variant == 0:
        return np.random.Generator(np.random.PCG64(seed))
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed, spawn_key=(variant,))))


@dataclass(frozen=True)
class Grid:
    """Search grid lam_i = lam0 + i*dlam (i < nlam), theta_j = th0 + j*dth deg (j < nth).

    The descriptor crosses the C boundary as float32 fields; node values are
    lam0 + i*dlam evaluated in float64 from those float32 fields, then rounded
    to float32.
    """
    lam0: float
    dlam: float
    nlam: int
    th0_deg: float
    dth_deg: float
    nth: int

    @property
    def size(self) -> int:
        return self.nlam * self.nth

    def lam_node(self, i: int) -> float:
        return float(np.float32(float(np.float32(self.lam0)) + i * float(np.float32(self.dlam))))

    def th_node(self, j: int) -> float:
        return float(np.float32(float(np.float32(self.th0_deg)) + j * float(np.float32(self.dth_deg))))


# 11 scales 0.96..1.04 x 11 rotations -1..1 deg (121 candidates per frame)
GRID_C1 = Grid(0.96, 0.008, 11, -1.0, 0.2, 11)
# 41 scales 0.9..1.1 step 0.005 x 41 rotations -5..5 deg step 0.25 (1681 per frame)
GRID_FULL = Grid(0.9, 0.005, 41, -5.0, 0.25, 41)


def fingerprint_field(H: int, W: int, rng: np.random.Generator, sigma: float = 0.02) -> np.ndarray:
    return (rng.standard_normal((H, W)) * sigma).astype(np.float32)


def content_field(H: int, W: int, rng: np.random.Generator, blur_sigma: float = 8.0,
                  lo: float = 16.0, hi: float = 240.0) -> np.ndarray:
    z = rng.standard_normal((H, W))
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.rfftfreq(W)[None, :]
    gain = np.exp(-2.0 * np.pi ** 2 * blur_sigma ** 2 * (fy ** 2 + fx ** 2))
    z = np.fft.irfft2(np.fft.rfft2(z) * gain, s=(H, W))
    z -= z.min()
    z /= max(z.max(), 1e-300)
    return lo + (hi - lo) * z


def sensor_frame(content: np.ndarray, K: np.ndarray, rng: np.random.Generator,
                 noise_sigma: float = 2.0) -> np.ndarray:
    return content * (1.0 + K.astype(np.float64)) + rng.standard_normal(content.shape) * noise_sigma


def stabilise(O: np.ndarray, lam: float, theta_deg: float, sy: float, sx: float) -> np.ndarray:
    """S(q) = O(lam*Rot(theta)(q-c) + c + s), bilinear, edge-replicated."""
    H, W = O.shape
    cy, cx = (H - 1) / 2.0, (W - 1) / 2.0
    th = np.deg2rad(theta_deg)
    ct, st = np.cos(th), np.sin(th)
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64) - cy, np.arange(W, dtype=np.float64) - cx,
                         indexing="ij")
    px = lam * (ct * xx - st * yy) + cx + sx
    py = lam * (st * xx + ct * yy) + cy + sy
    return ndimage.map_coordinates(O, [py, px], order=1, mode="nearest")


def quantise(x: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(x), 0, 255).astype(np.uint8)


def make_frames(K: np.ndarray, planted: np.ndarray, config: int, variant: int = 0) -> np.ndarray:
    """One stabilised uint8 frame per planted (lam, theta_deg, sy, sx) row."""
    H, W = K.shape
    rc = rng_for(config, STREAM_CONTENT, variant)
    rn = rng_for(config, STREAM_NOISE, variant)
    out = np.empty((len(planted), H, W), np.uint8)
    for f, (lam, th, sy, sx) in enumerate(planted):
        O = sensor_frame(content_field(H, W, rc), K, rn)
        out[f] = quantise(stabilise(O, lam, th, sy, sx))
    return out


def snap_windows(grid: Grid, centres: np.ndarray, ks: np.ndarray) -> np.ndarray:
    """Per-frame inclusive index windows [lam_lo, lam_hi, th_lo, th_hi].

    Each window is +-k grid steps around the node nearest to the given centre
    (lam, theta_deg); it is shifted, never clipped, to stay inside the grid, so
    it always holds exactly (2k+1)^2 candidates (or the whole axis if smaller).
    A negative k means the full grid.
    """
    out = np.empty((len(centres), 4), np.int32)
    lam0, dlam = float(np.float32(grid.lam0)), float(np.float32(grid.dlam))
    th0, dth = float(np.float32(grid.th0_deg)), float(np.float32(grid.dth_deg))
    for f, ((lam, th), k) in enumerate(zip(centres, ks)):
        if k < 0:
            out[f] = (0, grid.nlam - 1, 0, grid.nth - 1)
            continue
        row = []
        for v, v0, dv, n in ((lam, lam0, dlam, grid.nlam), (th, th0, dth, grid.nth)):
            c = int(np.clip(np.rint((v - v0) / dv), 0, n - 1))
            if 2 * k + 1 >= n:
                lo, hi = 0, n - 1
            else:
                lo, hi = c - k, c + k
                if lo < 0:
                    lo, hi = 0, 2 * k
                if hi > n - 1:
                    lo, hi = n - 1 - 2 * k, n - 1
            row += [lo, hi]
        out[f] = row
    return out


@dataclass
class Workload:
    name: str
    frames: np.ndarray                 # uint8 [F, H, W]
    fingerprints: list                 # float32 [H, W] each
    frame_fp: np.ndarray               # int [F]: fingerprint that generated the frame
    planted: np.ndarray                # float64 [F, 4]: lam, theta_deg, sy, sx
    grid: Grid
    windows: np.ndarray | None = None  # int32 [F, 4] or None (full grid)
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.frames.shape


def _draw_planted(rng, F, lam_rng, th_rng, s_max, grid: Grid | None, on_grid: bool):
    out = np.empty((F, 4))
    for f in range(F):
        if on_grid:
            lam = grid.lam_node(int(rng.integers(0, grid.nlam)))
            th = grid.th_node(int(rng.integers(0, grid.nth)))
        else:
            lam = rng.uniform(*lam_rng)
            th = rng.uniform(*th_rng)
        sy = int(rng.integers(-s_max, s_max + 1))
        sx = int(rng.integers(-s_max, s_max + 1))
        out[f] = (lam, th, sy, sx)
    return out


_DEFAULTS = {
    1: dict(H=256, W=256, F=4, grid=GRID_C1, lam=(0.96, 1.04), th=(-1.0, 1.0), s=8),
    2: dict(H=1080, W=1920, F=30, grid=GRID_FULL, lam=(0.9, 1.1), th=(-5.0, 5.0), s=64),
    3: dict(H=1080, W=1920, F=256, grid=GRID_FULL, lam=(0.9, 1.1), th=(-5.0, 5.0), s=64),
    4: dict(H=2160, W=3840, F=32, grid=GRID_FULL, lam=(0.9, 1.1), th=(-5.0, 5.0), s=64),
}


def make_workload(config: int, *, H: int | None = None, W: int | None = None, F: int | None = None,
                  on_grid: bool = False, grid: Grid | None = None, s_max: int | None = None,
                  frames: bool = True) -> Workload:
    """Build workload `config` (1..4), optionally at a reduced size.

    config 1: 256x256, 4 frames, 11x11 grid.      config 2: 1080p, 30 frames, 41x41 grid.
    config 3: 1080p, 256 frames, random-walk parameters and +-k warm-start windows.
    config 4: 2160x3840, 32 frames, half of them from an independent fingerprint.
    """
    d = dict(_DEFAULTS[config])
    H = H or d["H"]
    W = W or d["W"]
    F = F if F is not None else d["F"]
    grid = grid or d["grid"]
    s_max = d["s"] if s_max is None else s_max
    K = fingerprint_field(H, W, rng_for(config, STREAM_K))
    rt = rng_for(config, STREAM_TRANSFORM)
    windows = None
    fps = [K]
    frame_fp = np.zeros(F, np.int64)
    if config == 3:
        planted = np.empty((F, 4))
        lam, th = rt.uniform(0.95, 1.05), rt.uniform(-2.5, 2.5)
        for f in range(F):
            if f:
                lam = float(np.clip(lam + rt.normal(0, 0.003), d["lam"][0], d["lam"][1]))
                th = float(np.clip(th + rt.normal(0, 0.15), d["th"][0], d["th"][1]))
            planted[f] = (lam, th, int(rt.integers(-s_max, s_max + 1)), int(rt.integers(-s_max, s_max + 1)))
        ks = rt.integers(2, 11, size=F)
        ks[0] = -1                       # frame 0: full grid (no previous estimate)
        centres = np.vstack([planted[:1, :2], planted[:-1, :2]])
        windows = snap_windows(grid, centres, ks)
    else:
        planted = _draw_planted(rt, F, d["lam"], d["th"], s_max, grid, on_grid)
    if config == 4:
        K2 = fingerprint_field(H, W, rng_for(config, STREAM_K, variant=1))
        fps = [K, K2]
        frame_fp[F // 2:] = 1
    if frames:
        out = np.empty((F, H, W), np.uint8)
        for p, Kp in enumerate(fps):
            idx = np.nonzero(frame_fp == p)[0]
            if len(idx):
                out[idx] = make_frames(Kp, planted[idx], config, variant=p)
    else:
        out = np.empty((0, H, W), np.uint8)
    name = {1: "plain-256", 2: "plain-1080p", 3: "batched-1080p", 4: "precision-4k"}[config]
    return Workload(name=name, frames=out, fingerprints=[K] if config == 4 else fps,
                    frame_fp=frame_fp, planted=planted, grid=grid, windows=windows,
                    meta=dict(config=config, on_grid=on_grid, generated_by=list(range(len(fps)))))


@dataclass
class ServingQuery:
    qid: int
    arrival_s: float
    H: int
    W: int
    frames: np.ndarray | None  # uint8 [F, H, W]; None when the stream was made with materialise=False
    fp_ids: list              # fingerprint-bank ids to test, per resolution
    match: int                # bank id that generated the frames, or -1
    windows: np.ndarray       # int32 [F, 4]
    planted: np.ndarray
    pool: tuple = ()          # (H, W, source): the frame pool the frames come from
    pool_index: np.ndarray | None = None   # int [F]: frame f is pools[pool][pool_index[f]]


def make_query_stream(n_queries: int, *, rate_hz: float = 20.0,
                      resolutions=((720, 1280), (1080, 1920), (2160, 3840)),
                      frames_range=(8, 64), fps_range=(1, 16), bank_size: int = 16,
                      pool_frames: int = 64, grid: Grid = GRID_FULL, config: int = 5,
                      match_sources: int | None = None, materialise: bool = True):
    """Poisson query stream over per-resolution fingerprint banks and frame pools.

    To keep generation cheap, each resolution gets a pool of `pool_frames`
    stabilised frames per bank fingerprint that is actually drawn as a match
    (with `match_sources` set, only bank fingerprints 0..match_sources-1 can be
    the match); a query takes a contiguous run of a pool (wrapping around).
    Returns (queries, banks) where banks[(H, W)] is a list of float32 fingerprints.
    With materialise=False the queries carry no frame arrays, only their pool
    key and frame indices, and the return value is (queries, banks, pools)
    with pools[key] = uint8 [pool_frames, H, W].
    """
    ra = rng_for(config, STREAM_ARRIVALS)
    t = 0.0
    banks = {}
    pools = {}
    queries = []
    for q in range(n_queries):
        t += ra.exponential(1.0 / rate_hz)
        H, W = resolutions[int(ra.integers(0, len(resolutions)))]
        if (H, W) not in banks:
            banks[(H, W)] = [fingerprint_field(H, W, rng_for(config, STREAM_K, variant=1 + 1000 * H + b))
                             for b in range(bank_size)]
        F = int(ra.integers(frames_range[0], frames_range[1] + 1))
        P = int(ra.integers(fps_range[0], fps_range[1] + 1))
        fp_ids = sorted(ra.choice(bank_size, size=P, replace=False).tolist())
        match = int(fp_ids[int(ra.integers(0, P))]) if ra.random() < 0.5 else -1
        if match >= 0 and match_sources is not None and match >= match_sources:
            m = int(ra.integers(0, match_sources))
            if m not in fp_ids:
                fp_ids[fp_ids.index(match)] = m
                fp_ids.sort()
            match = m
        src = match if match >= 0 else bank_size  # bank_size = "no bank fingerprint"
        key = (H, W, src)
        if key not in pools:
            if src < bank_size:
                Kp = banks[(H, W)][src]
            else:
                # a camera outside the bank: its variant is disjoint from the
                # bank's 1 + 1000 H + b (b < bank_size <= 999)
                Kp = fingerprint_field(H, W, rng_for(config, STREAM_K, variant=5_000_000 + H))
            rt = rng_for(config, STREAM_TRANSFORM, variant=1 + 1000 * H + src)
            planted = np.empty((pool_frames, 4))
            lam, th = rt.uniform(0.95, 1.05), rt.uniform(-2.5, 2.5)
            for f in range(pool_frames):
                if f:
                    lam = float(np.clip(lam + rt.normal(0, 0.003), 0.9, 1.1))
                    th = float(np.clip(th + rt.normal(0, 0.15), -5.0, 5.0))
                planted[f] = (lam, th, int(rt.integers(-64, 65)), int(rt.integers(-64, 65)))
            pools[key] = (make_frames(Kp, planted, config, variant=1 + 1000 * H + src), planted)
        pf, pp = pools[key]
        start = int(ra.integers(0, pool_frames))
        idx = (start + np.arange(F)) % pool_frames
        ks = ra.integers(2, 11, size=F)
        centres = pp[(idx - 1) % pool_frames, :2]
        windows = snap_windows(grid, centres, ks)
        queries.append(ServingQuery(qid=q, arrival_s=t, H=H, W=W, frames=pf[idx] if materialise else None,
                                    fp_ids=fp_ids, match=match, windows=windows, planted=pp[idx], pool=key,
                                    pool_index=idx))
    if not materialise:
        return queries, banks, {k: v[0] for k, v in pools.items()}
    return queries, banks
