"""GPU parity of the frame-literal search (Sec. 3.2: warp the frame, extract
the residual per candidate) with the oracle, through the C ABI
(eis_grid_search_frames).

FP32 path: the arg-max candidate and its shift equal the oracle's and the PCE
is within 1e-3, unless the oracle's top two candidates lie within twice that
tolerance of each other (a near-tie), where the GPU's choice must score within
it under the oracle."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
FP32_TOL = 1e-3


@pytest.fixture(scope="module")
def prnu():
    import paper_2207_14507_gb300 as p
    p.build()
    return p


def _check(got, best, allp, frames, f, K0, weight):
    if int(got["cand_idx"]) == best["cand"]:
        assert (int(got["dy"]), int(got["dx"])) == (best["dy"], best["dx"])
        assert float(got["pce"]) == pytest.approx(best["pce"], rel=FP32_TOL)
        assert float(got["lam"]) == best["lam"] and float(got["th_deg"]) == best["th_deg"]
    else:
        o = oracle.score_literal(frames[f], K0, float(got["lam"]), float(got["th_deg"]), weight)
        assert o["pce"] >= best["pce"] * (1 - 2 * FP32_TOL), "GPU arg-max is not a near-tie of the oracle's"
        assert (int(got["dy"]), int(got["dx"])) == (o["dy"], o["dx"])


@pytest.mark.parametrize("weight", [True, False])
def test_literal_search_matches_oracle_256(prnu, weight):
    wl = synth.make_workload(1, on_grid=True)
    F = 2 if not weight else len(wl.frames)
    frames = wl.frames[:F]
    K = wl.fingerprints[0]
    K2 = synth.fingerprint_field(256, 256, np.random.default_rng(99))
    K0s = [oracle.fingerprint_term(K), oracle.fingerprint_term(K2)]
    best, allp = oracle.grid_search_literal(frames, K0s, wl.grid, weight_by_intensity=weight)
    with prnu.Context(0) as ctx:
        hs = [ctx.prnu_fingerprint_term(torch.from_numpy(k).to(DEV)) for k in (K, K2)]
        flags = prnu.PRNU_WEIGHT_BY_INTENSITY if weight else 0
        got = ctx.eis_grid_search_frames(torch.from_numpy(frames).to(DEV), hs, wl.grid, flags=flags)
        for f in range(F):
            for p in range(2):
                _check(got[f, p], best[f][p], allp, frames, f, K0s[p], weight)
            lam, th, sy, sx = wl.planted[f]
            assert (float(got[f, 0]["lam"]), float(got[f, 0]["th_deg"])) == (np.float32(lam), np.float32(th))
            assert (int(got[f, 0]["dy"]), int(got[f, 0]["dx"])) == (sy, sx)
            assert got[f, 1]["pce"] < 60


def test_literal_search_windows_pitch_and_chunks_1080p(prnu):
    """Full-HD frames with a row pitch, uneven windows: the oracle scores the
    GPU's best candidate one by one and checks it against the windows' best."""
    wl = synth.make_workload(2, F=2, on_grid=True)
    F, H, W = wl.frames.shape
    win = []
    for lam, th, _, _ in wl.planted:
        i = int(round((np.float32(lam) - np.float32(0.9)) / np.float32(0.005)))
        j = int(round((np.float32(th) + np.float32(5.0)) / np.float32(0.25)))
        win.append([max(i - 1, 0), min(i + 1, 40), max(j - 1, 0), min(j, 40)])
    win = np.array(win)
    K0 = oracle.fingerprint_term(wl.fingerprints[0])
    best, _ = oracle.grid_search_literal(wl.frames, [K0], wl.grid, windows=win)
    pitch = W + 64
    buf = np.zeros((F, H, pitch), np.uint8)
    buf[:, :, :W] = wl.frames
    with prnu.Context(0) as ctx:
        h = ctx.prnu_fingerprint_term(torch.from_numpy(wl.fingerprints[0]).to(DEV))
        d = torch.from_numpy(buf).to(DEV)
        # the binding takes the frame shape from the tensor: a [F, H, W] view with the row pitch
        view = d.as_strided((F, H, W), (H * pitch, pitch, 1))
        got = ctx.eis_grid_search_frames(view, [h], wl.grid, windows=win, pitch=pitch)
        for f in range(F):
            _check(got[f, 0], best[f][0], None, wl.frames, f, K0, True)
            assert (int(got[f, 0]["dy"]), int(got[f, 0]["dx"])) == tuple(wl.planted[f][2:].astype(int))


def test_literal_search_rejects_bad_arguments(prnu):
    wl = synth.make_workload(1, F=1, on_grid=True)
    with prnu.Context(0) as ctx:
        h = ctx.prnu_fingerprint_term(torch.from_numpy(wl.fingerprints[0]).to(DEV))
        fr = torch.from_numpy(wl.frames).to(DEV)
        with pytest.raises(prnu.PrnuError) as e:
            ctx.eis_grid_search_frames(fr, [h], wl.grid, flags=prnu.PRNU_NORMALISE)
        assert e.value.code == prnu.PRNU_EINVAL
        with pytest.raises(prnu.PrnuError) as e:
            ctx.eis_grid_search_frames(fr, [h], wl.grid, pitch=100)
        assert e.value.code == prnu.PRNU_EINVAL


def test_literal_search_over_many_chunks_equals_one_chunk(prnu):
    """Under a small HBM budget the renders of one frame span many chunks; the
    best kept across chunks equals the single-chunk result bit for bit (PCE,
    node, shift; ties keep the lowest candidate index)."""
    wl = synth.make_workload(1, on_grid=True)
    frames = torch.from_numpy(wl.frames[:2])
    K2 = synth.fingerprint_field(256, 256, np.random.default_rng(99))
    res = []
    # 64 MB: a quarter of it holds about 58 renders of 256x256 (residual plus
    # warped frame, 0.53 MB), so each 121-candidate frame spans three chunks;
    # waves of 16 keep the search's spectra at 4 MB
    for budget in (0, 64 << 20):
        with prnu.Context(0, hbm_budget_bytes=budget) as ctx:
            t = ctx.prnu_get_tuning(256, 256)
            ctx.prnu_set_tuning(256, 256, t["col_width"], t["pairs_per_block"], 16, t["variant"], 0)
            hs = [ctx.prnu_fingerprint_term(torch.from_numpy(k).to(DEV)) for k in (wl.fingerprints[0], K2)]
            res.append(ctx.eis_grid_search_frames(frames.to(DEV), hs, wl.grid))
    assert np.array_equal(res[0], res[1])
