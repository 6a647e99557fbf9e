"""Failure detection on the GPU without a fault: the bounded device-side waits
of the compile-time-planned kernels run out and are reported.

The test hook PRNU_DEBUG_STALL_DEVICE_WAITS makes every such wait expect one
arrival more than will ever come (the column pass's TMA barrier, the persistent
kernel's dependency counts).  Each wait gives up after about a second, the
kernel raises the context's error flag and abandons its candidate.  A call
that returns its results to the host fails with PRNU_EDEVICE_ABORT itself; a
call that leaves them on the device returns, and the next call fails.  Either
way the context then works again and gives the same results as before.  This
holds for the wave launches, the persistent kernel and the one-graph launch
(persistent = 0, 1, 2).  In the query server's device-resident loop, a query
whose wave saw the flag fails at query_poll, and the next queries of that
size run in a fresh loop."""
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


def _setup(ctx, prnu):
    g = synth.Grid(0.99, 0.01, 2, -0.5, 0.5, 2)          # 4 candidates
    wl = synth.make_workload(1, F=1, grid=g)
    R = torch.empty((1, 256, 256), device=DEV)
    ctx.prnu_residual(torch.from_numpy(wl.frames).to(DEV), R)
    h = ctx.prnu_fingerprint_term(torch.from_numpy(wl.fingerprints[0]).to(DEV))
    return g, R, h


@pytest.mark.parametrize("persistent", [0, 1, 2])
def test_bounded_device_wait_runs_out_and_is_reported(prnu, persistent):
    with prnu.Context(0) as ctx:
        g, R, h = _setup(ctx, prnu)
        t = ctx.prnu_get_tuning(256, 256)
        ctx.prnu_set_tuning(256, 256, t["col_width"], t["pairs_per_block"], 4, 0, persistent)
        good = ctx.eis_grid_search(R, [h], g)
        # host results: the stalled call reports the abort itself
        ctx.prnu_debug_set(prnu.PRNU_DEBUG_STALL_DEVICE_WAITS, 1)
        with pytest.raises(prnu.PrnuError) as e:
            ctx.eis_grid_search(R, [h], g)
        assert e.value.code == prnu.PRNU_EDEVICE_ABORT
        ctx.prnu_debug_set(prnu.PRNU_DEBUG_STALL_DEVICE_WAITS, 0)
        again = ctx.eis_grid_search(R, [h], g)              # the context is usable again
        assert np.array_equal(again["cand_idx"], good["cand_idx"])
        np.testing.assert_allclose(again["pce"], good["pce"], rtol=1e-12)
        # device results: the stalled call returns, the next one reports
        out = torch.empty((1, 32), dtype=torch.uint8, device=DEV)
        ctx.prnu_debug_set(prnu.PRNU_DEBUG_STALL_DEVICE_WAITS, 1)
        ctx.eis_grid_search(R, [h], g, out=out)
        torch.cuda.synchronize()
        ctx.prnu_debug_set(prnu.PRNU_DEBUG_STALL_DEVICE_WAITS, 0)
        with pytest.raises(prnu.PrnuError) as e:
            ctx.eis_grid_search(R, [h], g, out=out)
        assert e.value.code == prnu.PRNU_EDEVICE_ABORT
        again = ctx.eis_grid_search(R, [h], g)
        np.testing.assert_allclose(again["pce"], good["pce"], rtol=1e-12)
        with pytest.raises(prnu.PrnuError) as e:
            ctx.prnu_debug_set(99, 1)
        assert e.value.code == prnu.PRNU_EINVAL


def test_server_device_loop_wait_runs_out_and_is_reported(prnu):
    with prnu.Context(0) as ctx:
        g, R, h = _setup(ctx, prnu)
        wl = synth.make_workload(1, F=1, grid=g)
        frames = torch.from_numpy(wl.frames).to(DEV)
        flags = prnu.PRNU_WEIGHT_BY_INTENSITY

        def serve():
            qid = ctx.query_submit(frames, [h], g, dtype=prnu.PRNU_F32, flags=flags)
            return ctx.query_poll(qid, 1, 1, timeout_us=120_000_000)

        good = serve()
        ctx.prnu_debug_set(prnu.PRNU_DEBUG_STALL_DEVICE_WAITS, 1)
        with pytest.raises(prnu.PrnuError) as e:
            serve()
        assert e.value.code == prnu.PRNU_EDEVICE_ABORT
        ctx.prnu_debug_set(prnu.PRNU_DEBUG_STALL_DEVICE_WAITS, 0)
        again = serve()                                      # a fresh loop for this size
        assert again.tobytes() == good.tobytes()
