"""Column-pass fingerprint modes give identical results.

The column pass multiplies each frame column spectrum by the fingerprint's
(Eq. 3, the cross-correlation by FFT).  Where the fingerprint strip comes
from is a launch choice only:
* mode 2 copies it by TMA into the strip buffer once the last forward stage
  has taken its inputs;
* mode 3 copies it, from the start, into a region of its own;
* mode 4 does the same with a region sized for FP16 bins.  A wave with an FP32
  fingerprint then takes the first mode-2/3 variant.

With the shared forward pass and FP16 fingerprints only, the split inverse
half runs a mode-4 kernel with more blocks per SM at 720p and 1080p.

Each bin's arithmetic is the same in all of them, so every PCE, arg-max node
and shift must match bit for bit.  The test covers every planned frame size,
FP32 and FP16 fingerprints, and the shared forward pass on and off."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
# (H, W): column variant indices of mode 2 and of mode 3/4 (the registry order
# of the compile-time-planned kernels)
MODES = {(256, 256): (0, 2), (720, 1280): (2, 0), (1080, 1920): (1, 0), (2160, 3840): (1, 0)}


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


@pytest.mark.parametrize("fp_dtype", ["f32", "f16"])
@pytest.mark.parametrize("H,W", sorted(MODES))
def test_fingerprint_modes_are_bit_identical(ctx, prnu, H, W, fp_dtype):
    wl = synth.make_workload(2, H=H, W=W, F=2, on_grid=True, s_max=min(16, H // 8))
    fps = [wl.fingerprints[0], synth.fingerprint_field(H, W, np.random.default_rng(77))]
    win = synth.snap_windows(wl.grid, wl.planted[:, :2], np.array([1, 1]))
    half = fp_dtype == "f16"
    frames = torch.from_numpy(wl.frames).to(DEV)
    R = torch.empty(frames.shape, dtype=torch.float16 if half else torch.float32, device=DEV)
    sc = torch.empty(2, device=DEV)
    ctx.prnu_residual(frames, R, scale=sc,
                      flags=prnu.PRNU_WEIGHT_BY_INTENSITY | (prnu.PRNU_NORMALISE if half else 0))
    hs = [ctx.prnu_fingerprint_term(torch.from_numpy(K).to(DEV), prnu.PRNU_F16 if half else prnu.PRNU_F32)
          for K in fps]
    t0 = ctx.prnu_get_tuning(H, W)
    out = {}
    try:
        for v in MODES[(H, W)]:
            for share in (0, 1):
                ctx.prnu_set_tuning(H, W, t0["col_width"], t0["pairs_per_block"], 8, v, 0, 1, share)
                ap = torch.empty((2, 2, wl.grid.size), dtype=torch.float64, device=DEV)
                res = ctx.eis_grid_search(R, hs, wl.grid, windows=win, scale=sc, all_pce=ap)
                torch.cuda.synchronize()
                out[(v, share)] = (res.tobytes(), ap.cpu().numpy())
    finally:
        ctx.prnu_set_tuning(H, W, t0["col_width"], t0["pairs_per_block"], t0["wave"], t0["variant"],
                            t0["persistent"], t0["streams"], t0["share_forward"])
        for h in hs:
            ctx.prnu_fingerprint_release(h)
    ref = out[(MODES[(H, W)][0], 0)]
    for key, (rb, ap) in out.items():
        assert rb == ref[0], key
        np.testing.assert_array_equal(ap, ref[1], err_msg=str(key))
    # the camera's own fingerprint finds every planted node and shift
    res = np.frombuffer(ref[0], dtype=prnu.RESULT_DTYPE).reshape(2, 2)
    for f in range(2):
        lam, th, sy, sx = wl.planted[f]
        assert (res[f, 0]["lam"], res[f, 0]["th_deg"]) == (np.float32(lam), np.float32(th))
        assert (res[f, 0]["dy"], res[f, 0]["dx"]) == (sy, sx)
