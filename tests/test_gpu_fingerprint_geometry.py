"""GPU parity of the fingerprint's resampling to a video geometry (Sec. 3)
with the oracle, through the C ABI (prnu_fingerprint_resize)."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def prnu():
    import paper_2207_14507_gb300 as p
    p.build()
    return p


def test_image_fingerprint_to_full_hd(prnu):
    """A 4000x3000 image fingerprint down-scaled by 0.48 (1920x1440) and
    cropped to the 1920x1080 centre band: every value within 1e-5 of the
    oracle's largest magnitude (FP32 sums of at most 36 weighted taps)."""
    K = np.random.default_rng(6).normal(0, 0.02, (3000, 4000))
    ref = oracle.fingerprint_resize(K, 0.48, 180, 0, 1080, 1920)
    with prnu.Context(0) as ctx:
        got = ctx.prnu_fingerprint_resize(torch.from_numpy(K.astype(np.float32)).to(DEV), 0.48, 180, 0, 1080,
                                          1920).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("scale,y0,x0,H,W", [(1.0, 7, 9, 60, 80), (1.5, 10, 3, 90, 150), (0.75, 0, 0, 54, 96)])
def test_resize_small_cases(prnu, scale, y0, x0, H, W):
    """Identity crop (exact), up-scaling, a pitched input."""
    K = np.random.default_rng(int(scale * 100)).standard_normal((72, 128))
    ref = oracle.fingerprint_resize(K, scale, y0, x0, H, W)
    with prnu.Context(0) as ctx:
        buf = torch.zeros((72, 160), dtype=torch.float32, device=DEV)
        buf[:, :128] = torch.from_numpy(K.astype(np.float32)).to(DEV)
        got = ctx.prnu_fingerprint_resize(buf[:, :128], scale, y0, x0, H, W).cpu().numpy()
    if scale == 1.0:
        np.testing.assert_array_equal(got, K.astype(np.float32)[y0:y0 + H, x0:x0 + W])
    else:
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-5 * np.max(np.abs(ref)))


def test_resize_rejects_bad_crops(prnu):
    with prnu.Context(0) as ctx:
        K = torch.zeros((100, 100), dtype=torch.float32, device=DEV)
        for args in ((0.5, 0, 0, 51, 50), (0.5, -1, 0, 10, 10), (0.001, 0, 0, 1, 1), (float("nan"), 0, 0, 1, 1)):
            with pytest.raises(prnu.PrnuError) as e:
                ctx.prnu_fingerprint_resize(K, *args)
            assert e.value.code == prnu.PRNU_EINVAL
