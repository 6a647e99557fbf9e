"""GPU parity of the wavelet-denoiser residual (Mihcak's denoiser, Sec. 2.2)
with the oracle, through the C ABI (prnu_residual_wavelet), and of the search
run on it.

FP32 residuals: every value within 1e-3 of the oracle's largest magnitude
(four levels of 8-tap sums in FP32 carry relative errors near 1e-6 of the
coarse bands' magnitudes, about 2000 grey levels; the shrinkage is
continuous); FP16 storage with PRNU_NORMALISE: within FP16 rounding of the
scaled oracle residual."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def prnu():
    import paper_2207_14507_gb300 as p
    p.build()
    return p


@pytest.mark.parametrize("weight", [True, False])
def test_wavelet_residual_matches_oracle_256(prnu, weight):
    wl = synth.make_workload(1, on_grid=True)
    F = len(wl.frames)
    with prnu.Context(0) as ctx:
        out = torch.empty((F, 256, 256), device=DEV)
        flags = prnu.PRNU_WEIGHT_BY_INTENSITY if weight else 0
        got = ctx.prnu_residual_wavelet(torch.from_numpy(wl.frames).to(DEV), out, 3.0, flags).cpu().numpy()
    for f in range(F):
        ref = oracle.prnu_residual_wavelet(wl.frames[f], 3.0, weight)
        assert np.max(np.abs(got[f] - ref)) <= 1e-3 * np.max(np.abs(ref))


def test_wavelet_residual_1080p_pitch_and_fp16(prnu):
    """A full-HD frame (1080 rows: mirrored up to 1088) with a row pitch, FP32
    and FP16 + PRNU_NORMALISE."""
    wl = synth.make_workload(2, F=1, on_grid=True)
    H, W = wl.frames.shape[1:]
    ref = oracle.prnu_residual_wavelet(wl.frames[0], 3.0, True)
    buf = np.zeros((1, H, W + 32), np.uint8)
    buf[0, :, :W] = wl.frames[0]
    with prnu.Context(0) as ctx:
        d = torch.from_numpy(buf).to(DEV)
        view = d.as_strided((1, H, W), (H * (W + 32), W + 32, 1))
        out = torch.empty((1, H, W), device=DEV)
        got = ctx.prnu_residual_wavelet(view, out, 3.0, pitch=W + 32).cpu().numpy()[0]
        assert np.max(np.abs(got - ref)) <= 1e-3 * np.max(np.abs(ref))
        out16 = torch.empty((1, H, W), dtype=torch.float16, device=DEV)
        sc = torch.empty(1, device=DEV)
        got16 = ctx.prnu_residual_wavelet(view, out16, 3.0, prnu.PRNU_WEIGHT_BY_INTENSITY | prnu.PRNU_NORMALISE,
                                          scale=sc, pitch=W + 32).float().cpu().numpy()[0]
    s_ref = 1.0 / np.sqrt(np.mean(ref * ref))
    assert float(sc[0]) == pytest.approx(s_ref, rel=1e-4)
    scaled = ref * s_ref
    assert np.max(np.abs(got16 - scaled)) <= 2e-3 * np.max(np.abs(scaled))


def test_search_on_wavelet_residuals_matches_oracle(prnu):
    """The grid search on the library's wavelet residuals finds the oracle's
    best node and shift on every planted frame, PCE within 1e-3."""
    wl = synth.make_workload(1, on_grid=True)
    F = len(wl.frames)
    K0 = oracle.fingerprint_term(wl.fingerprints[0])
    R = [oracle.prnu_residual_wavelet(f) for f in wl.frames]
    best, _ = oracle.grid_search(R, [K0], wl.grid)
    with prnu.Context(0) as ctx:
        out = torch.empty((F, 256, 256), device=DEV)
        ctx.prnu_residual_wavelet(torch.from_numpy(wl.frames).to(DEV), out, 3.0)
        h = ctx.prnu_fingerprint_term(torch.from_numpy(wl.fingerprints[0]).to(DEV))
        got = ctx.eis_grid_search(out, [h], wl.grid)
    for f in range(F):
        g, b = got[f, 0], best[f][0]
        assert int(g["cand_idx"]) == b["cand"] and (int(g["dy"]), int(g["dx"])) == (b["dy"], b["dx"])
        assert float(g["pce"]) == pytest.approx(b["pce"], rel=1e-3)


def test_wavelet_residual_rejects_bad_arguments(prnu):
    with prnu.Context(0) as ctx:
        fr = torch.zeros((1, 32, 32), dtype=torch.uint8, device=DEV)
        out = torch.empty((1, 32, 32), device=DEV)
        for sigma in (-1.0, float("nan")):
            with pytest.raises(prnu.PrnuError) as e:
                ctx.prnu_residual_wavelet(fr, out, sigma)
            assert e.value.code == prnu.PRNU_EINVAL
        small = torch.zeros((1, 8, 32), dtype=torch.uint8, device=DEV)
        with pytest.raises(prnu.PrnuError) as e:
            ctx.prnu_residual_wavelet(small, torch.empty((1, 8, 32), device=DEV), 3.0)
        assert e.value.code == prnu.PRNU_EINVAL
        ctx.prnu_residual_wavelet(fr, out, 3.0)
        assert float(out.abs().max()) == 0.0     # a constant frame has no residual


def test_wavelet_residual_in_chunks_equals_one_chunk(prnu):
    """An 8 MB budget leaves room for about three 256x256 frames of scratch,
    so four frames run in two chunks (and PRNU_NORMALISE recomputes each chunk
    after the scales are known): the output equals the one-chunk run bit for
    bit."""
    wl = synth.make_workload(1, on_grid=True)
    F = len(wl.frames)
    outs = []
    for budget in (0, 8 << 20):
        with prnu.Context(0, hbm_budget_bytes=budget) as ctx:
            out = torch.empty((F, 256, 256), dtype=torch.float16, device=DEV)
            sc = torch.empty(F, device=DEV)
            ctx.prnu_residual_wavelet(torch.from_numpy(wl.frames).to(DEV), out, 3.0,
                                      prnu.PRNU_WEIGHT_BY_INTENSITY | prnu.PRNU_NORMALISE, scale=sc)
            outs.append((out.cpu().numpy(), sc.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
