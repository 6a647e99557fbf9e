"""Continuous-batching server (query_submit / query_poll) through the C ABI.

A query's results must not depend on what it was batched with: every query is
run alone and inside a concurrent mix of queries of other sizes, storage
types and frame locations, and the two runs must agree (the same kernels run
on the same inputs, so the PCE values are expected to be identical; the test
holds them to 1e-9 relative)."""
import time

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


def _mk(config, H, W, F, seed_grid, P=2, match=0, dtype=None, host=False):
    g = synth.Grid(0.97, 0.01, 7, -1.5, 0.5, 7)
    wl = synth.make_workload(config, H=H, W=W, F=F, grid=g, on_grid=True, s_max=12)
    rng = np.random.default_rng(seed_grid)
    fps = [wl.fingerprints[0]] + [synth.fingerprint_field(H, W, rng) for _ in range(P - 1)]
    if match != 0:
        fps = fps[1:] + fps[:1]
    wins = np.array([[int(rng.integers(0, 3)), int(rng.integers(4, 7)), int(rng.integers(0, 3)),
                      int(rng.integers(4, 7))] for _ in range(F)], np.int32)
    frames = torch.from_numpy(wl.frames)
    frames = frames.pin_memory() if host else frames.to(DEV)
    return dict(wl=wl, fps=fps, windows=wins, frames=frames, dtype=dtype, g=g)


def _handles(ctx, prnu, q):
    fpd = prnu.PRNU_F32 if q["dtype"] in (None, prnu.PRNU_F32) else prnu.PRNU_F16
    return [ctx.prnu_fingerprint_term(torch.from_numpy(K).to(DEV), fpd) for K in q["fps"]]


def _submit(ctx, prnu, q, hs):
    dt = prnu.PRNU_F32 if q["dtype"] is None else q["dtype"]
    flags = prnu.PRNU_WEIGHT_BY_INTENSITY | (0 if dt == prnu.PRNU_F32 else prnu.PRNU_NORMALISE)
    return ctx.query_submit(q["frames"], hs, q["g"], windows=q["windows"], dtype=dt, flags=flags)


def _same(a, b):
    assert np.array_equal(a["cand_idx"], b["cand_idx"])
    assert np.array_equal(a["dy"], b["dy"]) and np.array_equal(a["dx"], b["dx"])
    np.testing.assert_allclose(a["pce"], b["pce"], rtol=1e-9, atol=0)


def test_served_query_equals_eis_grid_search(prnu):
    with prnu.Context(0) as ctx:
        q = _mk(1, 256, 256, 3, 1)
        hs = _handles(ctx, prnu, q)
        qid = _submit(ctx, prnu, q, hs)
        served = ctx.query_poll(qid, 3, 2, timeout_us=60_000_000)
        R = torch.empty((3, 256, 256), device=DEV)
        ctx.prnu_residual(q["frames"], R)
        direct = ctx.eis_grid_search(R, hs, q["g"], windows=q["windows"])
        _same(served, direct)
        lat = ctx.query_latency(qid)
        assert 0 <= lat["queued_ms"] <= lat["total_ms"]
        # the oracle agrees on the matching fingerprint's arg-max
        Rh = [oracle.prnu_residual(f)[0] for f in q["wl"].frames]
        best, _ = oracle.grid_search(Rh, [oracle.fingerprint_term(q["fps"][0])], q["g"], windows=q["windows"])
        for f in range(3):
            assert served[f, 0]["cand_idx"] == best[f][0]["cand"]
            assert served[f, 0]["pce"] == pytest.approx(best[f][0]["pce"], rel=1e-3)


def test_results_same_alone_and_in_the_mix(prnu):
    specs = [
        dict(config=1, H=256, W=256, F=3, seed=11),                                  # compile-time kernels
        dict(config=2, H=160, W=200, F=4, seed=12, host=True),                      # generic kernels, host frames
        dict(config=1, H=256, W=256, F=2, seed=13, P=3, match=1, dtype="f16"),      # FP16 storage
        dict(config=2, H=160, W=200, F=2, seed=14, dtype="bf16"),
        dict(config=1, H=256, W=256, F=5, seed=15, P=1),
    ]
    with prnu.Context(0) as ctx:
        qs = []
        for s in specs:
            dt = {None: None, "f16": prnu.PRNU_F16, "bf16": prnu.PRNU_BF16}[s.get("dtype")]
            q = _mk(s["config"], s["H"], s["W"], s["F"], s["seed"], P=s.get("P", 2), match=s.get("match", 0),
                    dtype=dt, host=s.get("host", False))
            q["hs"] = _handles(ctx, prnu, q)
            q["P"] = s.get("P", 2)
            qs.append(q)
        alone = []
        for q in qs:
            qid = _submit(ctx, prnu, q, q["hs"])
            alone.append(ctx.query_poll(qid, q["wl"].frames.shape[0], q["P"], timeout_us=60_000_000))
        # the mix: everything submitted at once, twice over, so that waves span queries
        ids = [_submit(ctx, prnu, q, q["hs"]) for q in qs + qs]
        mixed = [ctx.query_poll(i, q["wl"].frames.shape[0], q["P"], timeout_us=120_000_000)
                 for i, q in zip(ids, qs + qs)]
        for k, q in enumerate(qs + qs):
            _same(alone[k % len(qs)], mixed[k])
        st = ctx.prnu_server_stats_get()
        assert st["queries_done"] == 3 * len(qs)
        per_query = [q["P"] * sum((w[1] - w[0] + 1) * (w[3] - w[2] + 1) for w in q["windows"]) for q in qs]
        assert st["candidates_done"] == 3 * sum(per_query)


def test_admission_waits_for_memory(prnu):
    """A budget with room for one 1080p query at a time (after the twiddles,
    the fingerprint spectrum and a 16-candidate workspace): later queries are
    admitted as earlier ones free their memory, and every query completes with
    the same results."""
    budget = 200 << 20
    with prnu.Context(0, hbm_budget_bytes=budget) as ctx:
        t = ctx.prnu_get_tuning(1080, 1920)
        ctx.prnu_set_tuning(1080, 1920, t["col_width"], t["pairs_per_block"], 16, t["variant"])
        q = _mk(2, 1080, 1920, 4, 21, P=1)
        hs = _handles(ctx, prnu, q)
        ids = [_submit(ctx, prnu, q, hs) for _ in range(6)]
        outs = [ctx.query_poll(i, 4, 1, timeout_us=120_000_000) for i in ids]
        for o in outs[1:]:
            _same(outs[0], o)
        st = ctx.prnu_server_stats_get()
        assert st["queries_done"] == 6
        assert st["admitted_bytes_peak"] < 2 * 4 * 1080 * 1920 * 4     # never two queries at once


def test_poll_and_submit_errors(prnu):
    with prnu.Context(0) as ctx:
        q = _mk(1, 256, 256, 2, 31, P=1)
        hs = _handles(ctx, prnu, q)
        qid = _submit(ctx, prnu, q, hs)
        early = ctx.query_poll(qid, 2, 1, timeout_us=0)      # EAGAIN -> None, or already done
        res = ctx.query_poll(qid, 2, 1, timeout_us=60_000_000)
        assert res is not None and (early is None or True)
        with pytest.raises(prnu.PrnuError) as e:
            ctx.query_poll(qid, 2, 1, timeout_us=0)
        assert e.value.code == prnu.PRNU_ENOTFOUND
        with pytest.raises(prnu.PrnuError) as e:
            ctx.query_submit(q["frames"], [hs[0] + 1000], q["g"])
        assert e.value.code == prnu.PRNU_ENOTFOUND
        bad = torch.zeros((1, 64, 70), dtype=torch.uint8, device=DEV)
        with pytest.raises(prnu.PrnuError) as e:
            ctx.query_submit(bad, hs, q["g"])
        assert e.value.code == prnu.PRNU_EINVAL
    with prnu.Context(0, hbm_budget_bytes=64 << 20) as small:
        # 16 full-HD frames: their residuals alone (66 MB) exceed the budget,
        # whatever wave the budget leaves room for
        big = torch.zeros((16, 1080, 1920), dtype=torch.uint8, device=DEV)
        K = torch.zeros((1080, 1920), device=DEV)
        h = small.prnu_fingerprint_term(K)
        with pytest.raises(prnu.PrnuError) as e:
            small.query_submit(big, [h], synth.GRID_FULL)
        assert e.value.code == prnu.PRNU_ENOMEM
