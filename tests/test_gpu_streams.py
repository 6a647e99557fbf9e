"""Two-stream waves (tuning field `streams`) give the same results as one
stream, bit for bit: the waves only change which stream and which half of the
workspace run them."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def prnu():
    import paper_2207_14507_gb300 as p
    p.build()
    return p


@pytest.mark.parametrize("shape", [(256, 256), (1080, 1920)])
def test_two_stream_waves_equal_one_stream(prnu, shape):
    cfg = 1 if shape == (256, 256) else 2
    wl = synth.make_workload(cfg, F=4 if cfg == 1 else 1)
    F, H, W = wl.frames.shape
    win = None if cfg == 1 else np.array([[10, 20, 10, 20]])    # 121 candidates
    res = []
    with prnu.Context(0) as ctx:
        fr = torch.from_numpy(wl.frames).to(DEV)
        R = torch.empty((F, H, W), device=DEV)
        ctx.prnu_residual(fr, R)
        h = ctx.prnu_fingerprint_term(torch.from_numpy(wl.fingerprints[0]).to(DEV))
        t = ctx.prnu_get_tuning(H, W)
        for streams in (1, 2, 2):
            ctx.prnu_set_tuning(H, W, t["col_width"], t["pairs_per_block"], 16, t["variant"], 0, streams)
            assert ctx.prnu_get_tuning(H, W)["streams"] == streams
            res.append(ctx.eis_grid_search(R, [h], wl.grid, windows=win))
    assert np.array_equal(res[0], res[1]) and np.array_equal(res[0], res[2])
