"""pce_score_noalloc: the aligned-pair PCE for callers that cannot allocate
device memory.  It must agree with pce_score (the allocating entry point)
within the FP32 tolerance of the other parity tests, on consecutive calls that
reuse its shared static scratch.  Collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-3
DEV = "cuda:0"


@pytest.fixture(scope="module")
def prnu():
    import paper_2207_14507_gb300 as p
    p.build()
    return p


def _pair(H, W, seed, gain=30.0):
    rng = np.random.default_rng(seed)
    K = (rng.standard_normal((H, W)) * 0.02).astype(np.float32)
    s = (int(rng.integers(-H // 2, H // 2)), int(rng.integers(-W // 2, W // 2)))
    X = (rng.standard_normal((H, W)) + gain * np.roll(K, shift=(-s[0], -s[1]), axis=(0, 1))).astype(np.float32)
    return torch.from_numpy(X).to(DEV), torch.from_numpy(K).to(DEV), s


def _reference(prnu, X, K):
    with prnu.Context(0) as ctx:
        h = ctx.prnu_fingerprint_term(K)
        r = ctx.pce_score(X, h)
        ctx.prnu_fingerprint_release(h)
    return r


def test_two_calls_in_a_row_match_pce_score(prnu):
    # the last pair is weak on purpose: its correlation maximum is a noise
    # peak, not the planted shift, and both entry points must still agree
    cases = [(_pair(256, 320, 1), True), (_pair(720, 1280, 2), True), (_pair(64, 48, 3, gain=3.0), False)]
    for (X, K, s), strong in cases:
        ref = _reference(prnu, X, K)
        if strong:
            assert (ref["dy"], ref["dx"]) == s
        for _call in range(2):
            got = prnu.pce_score_noalloc(X, K)
            assert (got["dy"], got["dx"]) == (ref["dy"], ref["dx"])
            assert got["pce"] == pytest.approx(ref["pce"], rel=FP32_TOL)
            assert got["peak"] == pytest.approx(ref["peak"], rel=FP32_TOL)


def test_square_frame_and_fingerprint_offset(prnu):
    """H == W (both FFT lengths share one size, so the two twiddle tables have
    the same length), and a fingerprint with a DC offset: the mean is removed
    inside, so K + 0.5 scores as K does."""
    X, K, s = _pair(1024, 1024, 7)
    ref = _reference(prnu, X, K)
    assert (ref["dy"], ref["dx"]) == s
    for _call in range(2):
        got = prnu.pce_score_noalloc(X, K)
        assert (got["dy"], got["dx"]) == s
        assert got["pce"] == pytest.approx(ref["pce"], rel=FP32_TOL)
        off = prnu.pce_score_noalloc(X, K + 0.5)
        assert (off["dy"], off["dx"]) == s
        assert off["pce"] == pytest.approx(ref["pce"], rel=FP32_TOL)


def test_rejects_mismatched_inputs(prnu):
    X, K, _ = _pair(128, 160, 9)
    with pytest.raises(prnu.PrnuError):
        prnu.pce_score_noalloc(X, K[:, :80].contiguous())
    with pytest.raises(prnu.PrnuError):
        prnu.pce_score_noalloc(X, K.half())
    with pytest.raises(prnu.PrnuError):
        prnu.pce_score_noalloc(X, K.t().contiguous().t())
    # through the C ABI: a host pointer is refused before any kernel runs
    import ctypes
    host = np.zeros((128, 160), np.float32)
    code = prnu.lib().pce_score_noalloc(ctypes.c_void_p(X.data_ptr()), host.ctypes.data_as(ctypes.c_void_p),
                                        128, 160, None, None, None, None, None)
    assert code == prnu.PRNU_EINVAL


def test_rejects_frames_beyond_the_limit(prnu):
    X = torch.zeros((1080, 1920), device=DEV)
    with pytest.raises(prnu.PrnuError) as e:
        prnu.pce_score_noalloc(X, X)
    assert e.value.code == prnu.PRNU_EINVAL
    # the scratch is still usable afterwards
    X, K, s = _pair(128, 160, 5)
    got = prnu.pce_score_noalloc(X, K)
    assert (got["dy"], got["dx"]) == s
