"""The seeded workload generator shared by the oracle and the CUDA path (it
holds none of the method's arithmetic): determinism, the statistics the
workload recipes state, the stabilisation convention, the warm-start windows."""
import numpy as np
import pytest

import synth
from synth import generate as gen


def test_workloads_are_reproducible():
    a, b = synth.make_workload(1), synth.make_workload(1)
    assert np.array_equal(a.frames, b.frames) and np.array_equal(a.planted, b.planted)
    assert np.array_equal(a.fingerprints[0], b.fingerprints[0])
    c = synth.make_workload(1, on_grid=True)
    assert not np.array_equal(a.planted, c.planted)


def test_recipe_statistics():
    wl = synth.make_workload(1)
    assert wl.frames.shape == (4, 256, 256) and wl.frames.dtype == np.uint8
    K = wl.fingerprints[0]
    assert K.dtype == np.float32 and abs(float(K.std()) - 0.02) < 5e-4 and abs(float(K.mean())) < 5e-4
    rng = gen.rng_for(1, 1)
    content = gen.content_field(256, 256, rng)
    assert content.min() == pytest.approx(16.0) and content.max() == pytest.approx(240.0)
    noise = gen.sensor_frame(np.full((256, 256), 100.0), np.zeros((256, 256)), gen.rng_for(1, 2)) - 100.0
    assert abs(float(noise.std()) - 2.0) < 0.05
    lam, th = wl.planted[:, 0], wl.planted[:, 1]
    assert np.all((lam >= 0.96) & (lam <= 1.04)) and np.all(np.abs(th) <= 1.0)
    assert np.all(np.abs(wl.planted[:, 2:]) <= 8) and np.all(wl.planted[:, 2:] == np.round(wl.planted[:, 2:]))


def test_stabilisation_convention():
    """S(q) = O(lam Rot(theta)(q - c) + c + s): the identity copies the frame,
    an integer shift s moves content so that S(q) = O(q + s)."""
    O = np.random.default_rng(0).uniform(0, 255, (40, 60))
    np.testing.assert_allclose(gen.stabilise(O, 1.0, 0.0, 0, 0), O, atol=1e-12)
    S = gen.stabilise(O, 1.0, 0.0, 3, -5)
    np.testing.assert_allclose(S[0:37, 5:60], O[3:40, 0:55], atol=1e-12)


def test_warm_start_windows():
    """Config 3: frame 0 searches the full grid; every other window holds
    exactly (2k + 1)^2 nodes, k in 2..10, inside the grid."""
    wl = synth.make_workload(3, H=64, W=96, F=40, frames=False)
    g, win = wl.grid, wl.windows
    assert tuple(win[0]) == (0, g.nlam - 1, 0, g.nth - 1)
    for lo_i, hi_i, lo_j, hi_j in win[1:]:
        n_i, n_j = hi_i - lo_i + 1, hi_j - lo_j + 1
        assert n_i == n_j and n_i % 2 == 1 and 5 <= n_i <= 21
        assert 0 <= lo_i and hi_i < g.nlam and 0 <= lo_j and hi_j < g.nth


def test_precision_workload_half_unmatched():
    """Config 4: the first half of the frames carries the fingerprint under
    test (the one fingerprint the workload exposes), the second half an
    independent one."""
    wl = synth.make_workload(4, H=64, W=96, F=8)
    assert list(wl.frame_fp) == [0] * 4 + [1] * 4 and len(wl.fingerprints) == 1
    assert wl.meta["generated_by"] == [0, 1]


def test_query_stream_without_frame_arrays_is_the_same_stream():
    q1, b1 = synth.make_query_stream(6, rate_hz=20.0, pool_frames=4, match_sources=1)
    q2, b2, pools = synth.make_query_stream(6, rate_hz=20.0, pool_frames=4, match_sources=1, materialise=False)
    for a, c in zip(q1, q2):
        assert c.frames is None
        assert np.array_equal(a.frames, pools[c.pool][c.pool_index])
        assert a.fp_ids == c.fp_ids and a.match == c.match and np.array_equal(a.windows, c.windows)


def test_out_of_bank_camera_differs_from_every_bank_fingerprint():
    qs, banks, pools = synth.make_query_stream(12, rate_hz=20.0, pool_frames=2, match_sources=1, materialise=False)
    for (H, W, src), frames in pools.items():
        if src < len(banks[(H, W)]):
            continue
        K = synth.fingerprint_field(H, W, synth.rng_for(5, gen.STREAM_K, variant=5_000_000 + H))
        for Kb in banks[(H, W)]:
            assert abs(np.corrcoef(K.ravel()[:100000], Kb.ravel()[:100000])[0, 1]) < 0.05
