"""GPU parity of the iterative correction (Sec. 3.2, Eq. 8) with the oracle,
through the C ABI (eis_correction).

Both sides search the same float32 node grids.  Where no near-tie sends the
two searches down different paths, the estimate, the shift and the iteration
count must be identical and the PCE within the FP32 path tolerance; where one
does, the GPU's estimate must score, under the oracle, within twice that
tolerance of the oracle's best."""
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


def _frames(planted, H=256, W=256):
    K = synth.fingerprint_field(H, W, synth.rng_for(1, 0))
    return K, synth.make_frames(K, np.asarray(planted, np.float64), 1)


def _check_pair(got, it, R, K0, lam0=1.0, th0=0.0, max_iter=3):
    best, iters, path = oracle.correction(R, K0, lam0=lam0, th0=th0, max_iter=max_iter, th_half1=5)
    if (float(got["lam"]), float(got["th_deg"])) == (best["lam"], best["th_deg"]):
        assert int(it) == iters
        assert (int(got["dy"]), int(got["dx"])) == (best["dy"], best["dx"])
        assert float(got["pce"]) == pytest.approx(best["pce"], rel=FP32_TOL)
    else:   # a near-tie took the searches apart: the GPU's estimate is as good under the oracle
        o = oracle.score(R, K0, float(got["lam"]), float(got["th_deg"]))
        assert o["pce"] >= best["pce"] * (1 - 2 * FP32_TOL)
        assert (int(got["dy"]), int(got["dx"])) == (o["dy"], o["dx"])
    return best


def test_correction_matches_oracle(prnu):
    lams, ths = oracle.correction_nodes(1.0, 0.0, 1, th_half1=5)
    planted = [(lams[7], ths[8], 3, -5), (1.0137, -0.262, -2, 4), (0.985, 0.41, 5, 1)]
    K, frames = _frames(planted)
    K2 = synth.fingerprint_field(256, 256, np.random.default_rng(77))
    with prnu.Context(0) as ctx:
        R = torch.empty((len(planted), 256, 256), device=DEV)
        ctx.prnu_residual(torch.from_numpy(frames).to(DEV), R)
        hs = [ctx.prnu_fingerprint_term(torch.from_numpy(k).to(DEV)) for k in (K, K2)]
        out, its = ctx.eis_correction(R, hs, th_half1=5)
        K0 = oracle.fingerprint_term(K)
        for f in range(len(planted)):
            Rf = oracle.prnu_residual(frames[f])[0]
            best = _check_pair(out[f, 0], its[f, 0], Rf, K0)
            assert abs(best["lam"] - planted[f][0]) <= 0.002 and abs(best["th_deg"] - planted[f][1]) <= 0.02
            assert 1 <= its[f, 1] <= 3 and out[f, 1]["pce"] < 60     # the other camera's fingerprint
        # a start estimate: the search begins around it (lattice frame, started on its node)
        init_l = np.array([[lams[7], 1.0]] * len(planted), np.float32)
        init_t = np.array([[ths[8], 0.0]] * len(planted), np.float32)
        out2, its2 = ctx.eis_correction(R, hs, init_lam=init_l, init_th=init_t, max_iter=2, th_half1=5)
        Rf = oracle.prnu_residual(frames[0])[0]
        _check_pair(out2[0, 0], its2[0, 0], Rf, K0, lam0=lams[7], th0=ths[8], max_iter=2)


def test_correction_rejects_bad_arguments(prnu):
    with prnu.Context(0) as ctx:
        R = torch.zeros((1, 256, 256), device=DEV)
        h = ctx.prnu_fingerprint_term(torch.zeros((256, 256), device=DEV))
        with pytest.raises(prnu.PrnuError) as e:
            ctx.eis_correction(R, [h], max_iter=0)
        assert e.value.code == prnu.PRNU_EINVAL
        with pytest.raises(prnu.PrnuError) as e:
            ctx.eis_correction(R, [h], init_lam=[-1.0])
        assert e.value.code == prnu.PRNU_EINVAL
        out, its = ctx.eis_correction(R, [h], max_iter=1, th_half1=2)   # zero residual: PCE 0, one iteration
        assert its[0, 0] == 1 and out[0, 0]["pce"] == 0.0


def test_correction_dense_first_grid_256(prnu):
    """The paper's dense first angle grid (Sec. 3.2: -5..5 degrees in steps of
    0.1, th_half1 = 50, 11 x 101 first-iteration nodes) at 256x256, with the
    oracle's exhaustive correction beside it."""
    planted = [(1.0137, -0.262, -2, 4), (0.9912, 2.34, 5, -3)]
    K, frames = _frames(planted)
    with prnu.Context(0) as ctx:
        R = torch.empty((len(planted), 256, 256), device=DEV)
        ctx.prnu_residual(torch.from_numpy(frames).to(DEV), R)
        h = ctx.prnu_fingerprint_term(torch.from_numpy(K).to(DEV))
        out, its = ctx.eis_correction(R, [h], th_half1=50)
        ctx.prnu_fingerprint_release(h)
    K0 = oracle.fingerprint_term(K)
    for f in range(len(planted)):
        Rf = oracle.prnu_residual(frames[f])[0]
        best, iters, _ = oracle.correction(Rf, K0, th_half1=50)
        _check_dense(out[f, 0], its[f, 0], Rf, K0, best, iters)
        assert abs(best["lam"] - planted[f][0]) <= 0.002 and abs(best["th_deg"] - planted[f][1]) <= 0.02


def test_correction_dense_first_grid_1080p(prnu):
    """The same at 1920x1080 (one frame, 1111 first-iteration nodes); the oracle
    scores each iteration's nodes in a pool of spawned processes."""
    wl = synth.make_workload(2, F=1, grid=synth.GRID_FULL)
    lam, th = 1.0214, -2.3311
    K = wl.fingerprints[0]
    frames = synth.make_frames(K, np.array([(lam, th, 17, -40)], np.float64), 2)
    with prnu.Context(0) as ctx:
        R = torch.empty((1, 1080, 1920), device=DEV)
        ctx.prnu_residual(torch.from_numpy(frames).to(DEV), R)
        h = ctx.prnu_fingerprint_term(torch.from_numpy(K).to(DEV))
        out, its = ctx.eis_correction(R, [h], th_half1=50)
        ctx.prnu_fingerprint_release(h)
    K0 = oracle.fingerprint_term(K)
    Rf = oracle.prnu_residual(frames[0])[0]
    with oracle.parallel.ScorePool(Rf, K0) as pool:
        best, iters, _ = oracle.correction(Rf, K0, th_half1=50, score_nodes=pool)
    _check_dense(out[0, 0], its[0, 0], Rf, K0, best, iters)
    assert abs(best["lam"] - lam) <= 0.002 and abs(best["th_deg"] - th) <= 0.02
    assert (int(out[0, 0]["dy"]), int(out[0, 0]["dx"])) == (17, -40)


def _check_dense(got, it, R, K0, best, iters):
    if (float(got["lam"]), float(got["th_deg"])) == (best["lam"], best["th_deg"]):
        assert int(it) == iters
        assert (int(got["dy"]), int(got["dx"])) == (best["dy"], best["dx"])
        assert float(got["pce"]) == pytest.approx(best["pce"], rel=FP32_TOL)
    else:   # a near-tie took the searches apart: the GPU's estimate is as good under the oracle
        o = oracle.score(R, K0, float(got["lam"]), float(got["th_deg"]))
        assert o["pce"] >= best["pce"] * (1 - 2 * FP32_TOL)
        assert (int(got["dy"]), int(got["dx"])) == (o["dy"], o["dx"])
