"""GPU parity of Algorithm 1 with supplied co-registration, and of the decision
mean(gamma) > tau (Sec. 3.2), with the oracle, through the C ABI
(eis_invert_video).

The segment is built so that every choice the algorithm makes has a wide
margin: the frames whose homography is right score far higher registered than
unwarped, and the frame whose homography is wrong was stabilised with the
identity.  The choices must then match the oracle's exactly; each frame's
correction is checked as in the correction parity test."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
FP32_TOL = 1e-3
TAU = 60.0     # these 256x256 segments: the null maximum over the searched nodes is far below


@pytest.fixture(scope="module")
def prnu():
    import paper_2207_14507_gb300 as p
    p.build()
    return p


def _homography(lam, th_deg, tx=0.0, ty=0.0):
    t = np.deg2rad(th_deg)
    c, s = np.cos(t), np.sin(t)
    return np.array([[lam * c, -lam * s, tx], [lam * s, lam * c, ty], [0.0, 0.0, 1.0]])


# anchor, three frames outside the first neighbourhood of (1, 0) with a close
# co-registration, one identity frame with a wrong co-registration
PLANTED = [(1.01, 0.2, 2, 1), (1.09, 4.3, -3, 2), (0.91, -4.6, 1, -4), (1.075, 2.9, 0, 3), (1.0, 0.0, 4, -2)]
HOMS = [np.eye(3)] + [_homography(p[0] + 0.003, p[1] - 0.05, 5.0, -2.0) for p in PLANTED[1:4]] + \
    [_homography(1.15, -7.0, 1.0, 1.0)]


def _segment(H=256, W=256):
    K = synth.fingerprint_field(H, W, synth.rng_for(1, 0))
    return K, synth.make_frames(K, np.asarray(PLANTED, np.float64), 1)


def test_invert_video_matches_oracle(prnu):
    K, frames = _segment()
    K0 = oracle.fingerprint_term(K)
    Rs = [oracle.prnu_residual(f)[0] for f in frames]
    ref = oracle.invert_video(Rs, K0, HOMS, max_iter=3, th_half1=5, tau=TAU)
    assert ref["from_reg"] == [False, True, True, True, False] and ref["decision"]
    K2 = synth.fingerprint_field(256, 256, np.random.default_rng(77))
    with prnu.Context(0) as ctx:
        R = torch.empty((len(PLANTED), 256, 256), device=DEV)
        ctx.prnu_residual(torch.from_numpy(frames).to(DEV), R)
        h, h2 = (ctx.prnu_fingerprint_term(torch.from_numpy(k).to(DEV)) for k in (K, K2))
        got = ctx.eis_invert_video(R, h, HOMS, max_iter=3, th_half1=5, tau=TAU)
        assert list(got["from_reg"]) == ref["from_reg"]
        for v in range(len(PLANTED)):
            g, b = got["best"][v], ref["best"][v]
            assert got["gamma"][v] == float(g["pce"])
            if (float(g["lam"]), float(g["th_deg"])) == (b["lam"], b["th_deg"]):
                assert (int(g["dy"]), int(g["dx"])) == (b["dy"], b["dx"])
                assert float(g["pce"]) == pytest.approx(b["pce"], rel=FP32_TOL)
            else:   # a near-tie: the GPU's node scores as well under the oracle
                o = oracle.score(Rs[v], K0, float(g["lam"]), float(g["th_deg"]))
                assert o["pce"] >= b["pce"] * (1 - 2 * FP32_TOL)
        assert got["mean"] == pytest.approx(float(np.mean(got["gamma"])), rel=1e-12)
        assert got["mean"] == pytest.approx(ref["mean"], rel=2 * FP32_TOL)
        assert got["decision"] == ref["decision"]

        # the corrections are eis_correction from the chosen starts, bit for bit
        lam0 = np.array([oracle.similarity_from_homography(HOMS[v])[0] if ref["from_reg"][v] else 1.0
                         for v in range(len(PLANTED))], np.float32)
        th0 = np.array([oracle.similarity_from_homography(HOMS[v])[1] if ref["from_reg"][v] else 0.0
                        for v in range(len(PLANTED))], np.float32)
        out, _ = ctx.eis_correction(R, [h], init_lam=lam0, init_th=th0, max_iter=3, th_half1=5)
        assert np.array_equal(out[:, 0]["pce"], got["gamma"])

        # no co-registration: every frame from (1, 0); the far frames are lost
        blind = ctx.eis_invert_video(R, h, None, max_iter=3, th_half1=5, tau=TAU)
        assert not blind["from_reg"].any() and blind["mean"] < got["mean"]
        out, _ = ctx.eis_correction(R, [h], max_iter=3, th_half1=5)
        assert np.array_equal(out[:, 0]["pce"], blind["gamma"])

        # another camera's fingerprint: no decision for it
        other = ctx.eis_invert_video(R, h2, HOMS, max_iter=3, th_half1=5, tau=TAU)
        assert not other["decision"] and max(other["gamma"]) < TAU
        ref2 = oracle.invert_video(Rs, oracle.fingerprint_term(K2), HOMS, max_iter=1, th_half1=5, tau=TAU)
        assert not ref2["decision"]


def test_invert_video_single_frame_and_bad_arguments(prnu):
    K, frames = _segment()
    with prnu.Context(0) as ctx:
        R = torch.empty((1, 256, 256), device=DEV)
        ctx.prnu_residual(torch.from_numpy(frames[:1]).to(DEV), R)
        h = ctx.prnu_fingerprint_term(torch.from_numpy(K).to(DEV))
        one = ctx.eis_invert_video(R, h, [np.eye(3)], max_iter=2, th_half1=5, tau=TAU)
        out, _ = ctx.eis_correction(R, [h], max_iter=2, th_half1=5)
        assert one["gamma"][0] == float(out[0, 0]["pce"]) and one["mean"] == one["gamma"][0]
        assert one["decision"] and not one["from_reg"][0]
        R2 = R.expand(2, 256, 256).contiguous()
        for bad in (np.zeros((3, 3)), np.array([[np.inf, 0, 0], [0, 1, 0], [0, 0, 1.0]])):
            with pytest.raises(prnu.PrnuError) as e:
                ctx.eis_invert_video(R2, h, [np.eye(3), bad], max_iter=1, th_half1=5)
            assert e.value.code == prnu.PRNU_EINVAL
        with pytest.raises(prnu.PrnuError) as e:
            ctx.eis_invert_video(R2, h, None, max_iter=0)
        assert e.value.code == prnu.PRNU_EINVAL
        with pytest.raises(prnu.PrnuError) as e:
            ctx.eis_invert_video(R2, h, None, tau=float("nan"))
        assert e.value.code == prnu.PRNU_EINVAL
