"""One forward pass shared by the fingerprints of a (frame, grid node).

Eq. 3 correlates one frame's warped residual with each candidate device's
fingerprint (Sec. 4 tests a video against several devices), so the warp, the
row FFT and the forward column FFT of a (frame, node) do not depend on the
fingerprint.  With share_forward = 1 (the default) the library runs them once
per (frame, node) and only the product and the inverse FFT per fingerprint;
every candidate's arithmetic is unchanged, so the results must equal those of
share_forward = 0 bit for bit: every PCE, every arg-max node, shift and peak.
Also through the query server, and against the FP64 oracle at 256x256."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SHAPES = [(256, 256), (720, 1280), (1080, 1920), (2160, 3840)]


@pytest.fixture(scope="module")
def prnu():
    import paper_2207_14507_gb300 as p
    p.build()
    return p


@pytest.fixture(scope="module")
def ctx(prnu):
    c = prnu.Context(0)
    yield c
    c.close()


def _fingerprints(wl, P):
    H, W = wl.frames.shape[1:]
    fps = [wl.fingerprints[0]]
    for p in range(1, P):
        fps.append(synth.fingerprint_field(H, W, np.random.default_rng(1000 + p)))
    return fps


def _search(ctx, prnu, wl, fps, windows, dtype, share, wave):
    H, W = wl.frames.shape[1:]
    half = dtype != torch.float32
    frames = torch.from_numpy(wl.frames).to(DEV)
    R = torch.empty(frames.shape, dtype=dtype, device=DEV)
    scale = torch.empty(frames.shape[0], device=DEV)
    ctx.prnu_residual(frames, R, scale=scale,
                      flags=prnu.PRNU_WEIGHT_BY_INTENSITY | (prnu.PRNU_NORMALISE if half else 0))
    hs = [ctx.prnu_fingerprint_term(torch.from_numpy(K).to(DEV), prnu.PRNU_F16 if half else prnu.PRNU_F32)
          for K in fps]
    t0 = ctx.prnu_get_tuning(H, W)
    try:
        ctx.prnu_set_tuning(H, W, t0["col_width"], t0["pairs_per_block"], wave, t0["variant"], 0, 1, share)
        allp = torch.empty((len(wl.frames), len(hs), wl.grid.size), dtype=torch.float64, device=DEV)
        res = ctx.eis_grid_search(R, hs, wl.grid, windows=windows, scale=scale, all_pce=allp)
        torch.cuda.synchronize()
    finally:
        ctx.prnu_set_tuning(H, W, t0["col_width"], t0["pairs_per_block"], t0["wave"], t0["variant"],
                            t0["persistent"], t0["streams"], t0["share_forward"])
        for h in hs:
            ctx.prnu_fingerprint_release(h)
    return res, allp.cpu().numpy()


@pytest.mark.parametrize("dtype", ["float32", "float16"])
@pytest.mark.parametrize("H,W", SHAPES)
def test_shared_forward_is_bit_identical(ctx, prnu, H, W, dtype):
    dt = getattr(torch, dtype)
    wl = synth.make_workload(2, H=H, W=W, F=2, on_grid=True, s_max=min(16, H // 8))
    fps = _fingerprints(wl, 3)
    win = synth.snap_windows(wl.grid, wl.planted[:, :2], np.array([1, 1]))       # 3 x 3 nodes per frame
    # waves of 8 candidates: rounded down to whole units of 3 (6), several waves per call
    res1, all1 = _search(ctx, prnu, wl, fps, win, dt, 1, 8)
    res0, all0 = _search(ctx, prnu, wl, fps, win, dt, 0, 8)
    np.testing.assert_array_equal(all1, all0)
    assert res1.tobytes() == res0.tobytes()
    # the camera's own fingerprint finds the planted node and shift; the others do not
    for f in range(2):
        lam, th, sy, sx = wl.planted[f]
        assert (res1[f, 0]["lam"], res1[f, 0]["th_deg"]) == (np.float32(lam), np.float32(th))
        assert (res1[f, 0]["dy"], res1[f, 0]["dx"]) == (sy, sx)
        assert res1[f, 1]["pce"] < 60 and res1[f, 2]["pce"] < 60


def test_shared_forward_matches_oracle_256(ctx, prnu):
    wl = synth.make_workload(1, F=2)
    fps = _fingerprints(wl, 2)
    win = np.array([[2, 6, 3, 7], [4, 8, 1, 5]], np.int32)
    res, got = _search(ctx, prnu, wl, fps, win, torch.float32, 1, 64)
    R = [oracle.prnu_residual(f)[0] for f in wl.frames]
    best, ref = oracle.grid_search(R, [oracle.fingerprint_term(K) for K in fps], wl.grid, windows=win)
    mask = ~np.isnan(ref)
    assert np.array_equal(mask, ~np.isnan(got))
    assert np.max(np.abs(got[mask] - ref[mask]) / np.abs(ref[mask])) <= 1e-3
    for f in range(2):      # the camera's own fingerprint: the oracle's arg-max node and shift
        b = best[f][0]
        assert res[f, 0]["cand_idx"] == b["cand"] and (res[f, 0]["dy"], res[f, 0]["dx"]) == (b["dy"], b["dx"])


def test_served_queries_share_and_match(ctx, prnu):
    """Queries of 3 fingerprints through query_submit: equal, bit for bit, to
    eis_grid_search with and without the shared forward pass."""
    wl = synth.make_workload(2, H=720, W=1280, F=3, on_grid=True, s_max=16)
    fps = _fingerprints(wl, 3)
    win = synth.snap_windows(wl.grid, wl.planted[:, :2], np.array([2, 1, 2]))
    hs = [ctx.prnu_fingerprint_term(torch.from_numpy(K).to(DEV), prnu.PRNU_F16) for K in fps]
    frames = torch.from_numpy(wl.frames).to(DEV)
    flags = prnu.PRNU_WEIGHT_BY_INTENSITY | prnu.PRNU_NORMALISE
    qids = [ctx.query_submit(frames, hs, wl.grid, windows=win, dtype=prnu.PRNU_F16, flags=flags) for _ in range(2)]
    served = [ctx.query_poll(q, 3, 3, timeout_us=-1) for q in qids]
    for h in hs:
        ctx.prnu_fingerprint_release(h)
    res1, _ = _search(ctx, prnu, wl, fps, win, torch.float16, 1, 64)
    res0, _ = _search(ctx, prnu, wl, fps, win, torch.float16, 0, 64)
    assert res1.tobytes() == res0.tobytes()
    for s in served:
        assert s.tobytes() == res1.tobytes()


def test_sharing_steps_aside_where_it_cannot_apply(ctx, prnu):
    """Sizes without compile-time-planned kernels, the persistent launch, and
    waves smaller than one unit run every candidate alone: the results equal
    the default path's (waves of shared units where it applies)."""
    # a size with no planned kernels: 240 x 320, three fingerprints
    wl = synth.make_workload(2, H=240, W=320, F=2, on_grid=True, s_max=8)
    fps = _fingerprints(wl, 3)
    win = synth.snap_windows(wl.grid, wl.planted[:, :2], np.array([1, 1]))
    r1, a1 = _search(ctx, prnu, wl, fps, win, torch.float32, 1, 8)
    r0, a0 = _search(ctx, prnu, wl, fps, win, torch.float32, 0, 8)
    assert r1.tobytes() == r0.tobytes()
    np.testing.assert_array_equal(a1, a0)
    # a planned size: waves of 2 candidates (smaller than a unit of 3), and the persistent launch
    wl = synth.make_workload(1, F=2, on_grid=True)
    fps = _fingerprints(wl, 3)
    win = synth.snap_windows(wl.grid, wl.planted[:, :2], np.array([1, 2]))
    ref, aref = _search(ctx, prnu, wl, fps, win, torch.float32, 1, 64)
    small, asmall = _search(ctx, prnu, wl, fps, win, torch.float32, 1, 2)
    assert small.tobytes() == ref.tobytes()
    np.testing.assert_array_equal(asmall, aref)
    t0 = ctx.prnu_get_tuning(256, 256)
    try:
        ctx.prnu_set_tuning(256, 256, t0["col_width"], t0["pairs_per_block"], 64, 0, 1, 1, 1)
        frames = torch.from_numpy(wl.frames).to(DEV)
        R = torch.empty(frames.shape, device=DEV)
        sc = torch.empty(2, device=DEV)
        ctx.prnu_residual(frames, R, scale=sc)
        hs = [ctx.prnu_fingerprint_term(torch.from_numpy(K).to(DEV)) for K in fps]
        ap = torch.empty((2, 3, wl.grid.size), dtype=torch.float64, device=DEV)
        pers = ctx.eis_grid_search(R, hs, wl.grid, windows=win, scale=sc, all_pce=ap)
        torch.cuda.synchronize()
        for h in hs:
            ctx.prnu_fingerprint_release(h)
    finally:
        ctx.prnu_set_tuning(256, 256, t0["col_width"], t0["pairs_per_block"], t0["wave"], t0["variant"],
                            t0["persistent"], t0["streams"], t0["share_forward"])
    np.testing.assert_allclose(ap.cpu().numpy(), aref, rtol=1e-5)
    assert np.array_equal(pers["cand_idx"], ref["cand_idx"])
    assert np.array_equal(pers["dy"], ref["dy"]) and np.array_equal(pers["dx"], ref["dx"])
