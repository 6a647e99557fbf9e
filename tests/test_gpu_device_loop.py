"""The query server's device-resident request loop (prnu_server_set_loop).

With PRNU_LOOP_DEVICE the waves of frame sizes with compile-time-planned
kernels are formed on the GPU.  A CUDA graph per size repeats a scheduler
kernel, the wave kernels (shared-forward or plain branch) and a completion
kernel that writes each finished query's arg-max to host-mapped memory.  The
kernels are those of the host loop, fed the same candidates, so every query's
results must equal the host loop's bit for bit.  That holds alone, in a mix
of sizes, storage types and fingerprint counts, across several waves per
query, with many queries finishing in one wave, and for a size without
planned kernels (which takes host waves inside the device mode)."""
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


def _query(H, W, F, P, half, seed, full_grid=False):
    if full_grid:
        g = synth.Grid(0.97, 0.01, 11, -1.5, 0.3, 11)
        wl = synth.make_workload(1, H=H, W=W, F=F, grid=g)
        wins = None
    else:
        g = synth.Grid(0.97, 0.01, 7, -1.5, 0.5, 7)
        wl = synth.make_workload(2, H=H, W=W, F=F, grid=g, on_grid=True, s_max=min(12, H // 8))
        rng = np.random.default_rng(seed)
        # windows around the planted node, of uneven half-widths 1-2
        wins = synth.snap_windows(g, wl.planted[:, :2], rng.integers(1, 3, size=F))
    rng = np.random.default_rng(1000 + seed)
    fps = [wl.fingerprints[0]] + [synth.fingerprint_field(H, W, rng) for _ in range(P - 1)]
    return dict(frames=torch.from_numpy(wl.frames).to(DEV), fps=fps, g=g, windows=wins, half=half, F=F, P=P)


def _serve(prnu, mode, queries, order=None):
    """Serve the queries (all submitted before the first poll) on a fresh
    context with the given loop; returns their results in submission order."""
    with prnu.Context(0) as ctx:
        ctx.prnu_server_set_loop(mode)
        ids = []
        for q in (queries if order is None else [queries[i] for i in order]):
            fpd = prnu.PRNU_F16 if q["half"] else prnu.PRNU_F32
            hs = [ctx.prnu_fingerprint_term(torch.from_numpy(K).to(DEV), fpd) for K in q["fps"]]
            dt = prnu.PRNU_F16 if q["half"] else prnu.PRNU_F32
            flags = prnu.PRNU_WEIGHT_BY_INTENSITY | (prnu.PRNU_NORMALISE if q["half"] else 0)
            ids.append((ctx.query_submit(q["frames"], hs, q["g"], windows=q["windows"], dtype=dt, flags=flags), q))
        out = [ctx.query_poll(i, q["F"], q["P"], timeout_us=300_000_000) for i, q in ids]
        stats = ctx.prnu_server_stats_get()
    return out, stats


MIX = [(256, 256, 3, 2, False, 1, True),      # planned, FP32, several waves per query
       (720, 1280, 2, 3, True, 2, False),     # planned, FP16, shared forward units
       (1080, 1920, 2, 1, True, 3, False),    # planned, FP16, plain branch
       (240, 320, 2, 2, False, 4, False),     # no planned kernels: host waves in device mode
       (256, 256, 2, 3, True, 5, True)]       # planned, FP16, shared units, several waves


def test_device_loop_equals_host_loop(prnu):
    qs = [_query(*m) for m in MIX]
    dev, st = _serve(prnu, prnu.PRNU_LOOP_DEVICE, qs)
    host, _ = _serve(prnu, prnu.PRNU_LOOP_HOST, qs)
    for d, h in zip(dev, host):
        assert d.tobytes() == h.tobytes()
    assert st["queries_done"] == len(qs) and st["server_launches"] > 0
    # the matching fingerprint finds every planted node and shift (the windowed queries)
    for q, d in zip(qs, dev):
        if q["windows"] is None:
            continue
        assert np.all(d[:, 0]["pce"] > 60)


def test_device_loop_alone_and_in_the_mix(prnu):
    qs = [_query(*m) for m in MIX]
    alone, _ = _serve(prnu, prnu.PRNU_LOOP_DEVICE, qs[1:2])
    mixed, _ = _serve(prnu, prnu.PRNU_LOOP_DEVICE, qs, order=[4, 0, 3, 1, 2])
    assert alone[0].tobytes() == mixed[3].tobytes()


def test_device_loop_many_small_queries(prnu):
    """48 one-frame 256x256 queries at once: many finish in the same wave and
    the loop relaunches across its wave budget; each equals eis_grid_search."""
    qs = [_query(256, 256, 1, 1 + (i % 3), bool(i % 2), 100 + i) for i in range(48)]
    dev, st = _serve(prnu, prnu.PRNU_LOOP_DEVICE, qs)
    host, _ = _serve(prnu, prnu.PRNU_LOOP_HOST, qs)
    for d, h in zip(dev, host):
        assert d.tobytes() == h.tobytes()
    assert st["candidates_done"] == sum(q["P"] * int(np.prod(q["windows"][:, 1] - q["windows"][:, 0] + 1) *
                                                     np.prod(q["windows"][:, 3] - q["windows"][:, 2] + 1))
                                        for q in qs)


def test_loop_mode_rules(prnu):
    with prnu.Context(0) as ctx:
        with pytest.raises(prnu.PrnuError) as e:
            ctx.prnu_server_set_loop(7)
        assert e.value.code == prnu.PRNU_EINVAL
        ctx.prnu_server_set_loop(prnu.PRNU_LOOP_DEVICE)
        q = _query(256, 256, 1, 1, False, 9)
        h = ctx.prnu_fingerprint_term(torch.from_numpy(q["fps"][0]).to(DEV))
        qid = ctx.query_submit(q["frames"], [h], q["g"], windows=q["windows"], dtype=prnu.PRNU_F32,
                               flags=prnu.PRNU_WEIGHT_BY_INTENSITY)
        ctx.query_poll(qid, 1, 1, timeout_us=60_000_000)
        ctx.prnu_server_set_loop(prnu.PRNU_LOOP_DEVICE)        # unchanged: fine
        with pytest.raises(prnu.PrnuError) as e:
            ctx.prnu_server_set_loop(prnu.PRNU_LOOP_HOST)      # the server has started
        assert e.value.code == prnu.PRNU_EINVAL


# ------------------------------------------------------------------ eis_grid_search in one graph launch

def _grid_search(ctx, prnu, wl, fps, windows, dtype, persistent, wave=64):
    H, W = wl.frames.shape[1:]
    half = dtype != torch.float32
    frames = torch.from_numpy(wl.frames).to(DEV)
    R = torch.empty(frames.shape, dtype=dtype, device=DEV)
    sc = torch.empty(frames.shape[0], device=DEV)
    ctx.prnu_residual(frames, R, scale=sc,
                      flags=prnu.PRNU_WEIGHT_BY_INTENSITY | (prnu.PRNU_NORMALISE if half else 0))
    hs = [ctx.prnu_fingerprint_term(torch.from_numpy(K).to(DEV), prnu.PRNU_F16 if half else prnu.PRNU_F32)
          for K in fps]
    t0 = ctx.prnu_get_tuning(H, W)
    try:
        ctx.prnu_set_tuning(H, W, t0["col_width"], t0["pairs_per_block"], wave, t0["variant"], persistent, 1,
                            t0["share_forward"])
        out = []
        for _ in range(2):   # the second call replays the graph built by the first
            allp = torch.empty((len(wl.frames), len(hs), wl.grid.size), dtype=torch.float64, device=DEV)
            res = ctx.eis_grid_search(R, hs, wl.grid, windows=windows, scale=sc, all_pce=allp)
            torch.cuda.synchronize()
            out.append((res.tobytes(), allp.cpu().numpy()))
    finally:
        ctx.prnu_set_tuning(H, W, t0["col_width"], t0["pairs_per_block"], t0["wave"], t0["variant"],
                            t0["persistent"], t0["streams"], t0["share_forward"])
        for h in hs:
            ctx.prnu_fingerprint_release(h)
    assert out[0][0] == out[1][0]
    return out[0]


@pytest.mark.parametrize("dtype", ["float32", "float16"])
@pytest.mark.parametrize("H,W", [(256, 256), (720, 1280), (1080, 1920), (2160, 3840)])
def test_grid_search_in_one_graph_launch_equals_waves(prnu, H, W, dtype):
    """prnu_tuning.persistent = 2 runs every wave of an eis_grid_search call in
    one graph launch (the device-resident loop over the call's work list):
    the same results as the wave launches, bit for bit, with one fingerprint
    (full grid at 256x256, several waves) and with three sharing forward units
    (windows)."""
    dt = getattr(torch, dtype)
    with prnu.Context(0) as ctx:
        if H == 256:
            wl = synth.make_workload(1, F=2)
            fps, win = [wl.fingerprints[0]], None
        else:
            wl = synth.make_workload(2, H=H, W=W, F=2, on_grid=True, s_max=min(16, H // 8))
            fps = [wl.fingerprints[0], synth.fingerprint_field(H, W, np.random.default_rng(3)),
                   synth.fingerprint_field(H, W, np.random.default_rng(4))]
            win = synth.snap_windows(wl.grid, wl.planted[:, :2], np.array([1, 2]))
        g_res, g_all = _grid_search(ctx, prnu, wl, fps, win, dt, 2)
        w_res, w_all = _grid_search(ctx, prnu, wl, fps, win, dt, 0)
    assert g_res == w_res
    np.testing.assert_array_equal(g_all, w_all)


def test_graph_launch_rebuilt_between_asynchronous_calls(prnu):
    """Two eis_grid_search calls with persistent = 2 and device outputs, back
    to back without a synchronisation, whose scale tensors differ: the second
    call rebuilds the graph while the first may still run (the old graph is
    destroyed only after its last launch).  Both equal the wave launches."""
    wl = synth.make_workload(1, F=2)
    with prnu.Context(0) as ctx:
        frames = torch.from_numpy(wl.frames).to(DEV)
        R = torch.empty((2, 256, 256), device=DEV)
        sc1 = torch.empty(2, device=DEV)
        ctx.prnu_residual(frames, R, scale=sc1, flags=prnu.PRNU_WEIGHT_BY_INTENSITY)
        sc2 = sc1.clone()
        h = ctx.prnu_fingerprint_term(torch.from_numpy(wl.fingerprints[0]).to(DEV))
        ref = ctx.eis_grid_search(R, [h], wl.grid, scale=sc1)
        t0 = ctx.prnu_get_tuning(256, 256)
        try:
            ctx.prnu_set_tuning(256, 256, t0["col_width"], t0["pairs_per_block"], 16, t0["variant"], 2)
            o1 = torch.empty((2, 32), dtype=torch.uint8, device=DEV)
            o2 = torch.empty((2, 32), dtype=torch.uint8, device=DEV)
            ctx.eis_grid_search(R, [h], wl.grid, scale=sc1, out=o1)
            ctx.eis_grid_search(R, [h], wl.grid, scale=sc2, out=o2)
            torch.cuda.synchronize()
        finally:
            ctx.prnu_set_tuning(256, 256, t0["col_width"], t0["pairs_per_block"], t0["wave"], t0["variant"],
                                t0["persistent"], t0["streams"], t0["share_forward"])
            ctx.prnu_fingerprint_release(h)
        for o in (o1, o2):
            assert o.cpu().numpy().tobytes() == ref.tobytes()


def test_correction_loop_on_the_device_equals_the_host_loop(prnu):
    """The iterative correction (Sec. 3.2): with persistent = 2 its loop runs
    on the device.  A kernel writes each iteration's work list (every active
    pair's window around its estimate), one graph launch scores it, and a
    kernel updates the estimates and drops converged pairs, with no host
    round trip until the end.  It must take the host loop's path: the same
    iteration counts and the same nodes and shifts, with PCE within 1e-5.
    The device forms the nodes' warp coefficients with its own double sincos,
    so a node may differ in the last bit.  Where a near-tie then picks
    another node, the two must score the same."""
    H, W = 720, 1280
    wl = synth.make_workload(2, H=H, W=W, F=3)
    fps = [wl.fingerprints[0], synth.fingerprint_field(H, W, np.random.default_rng(8))]
    lam0 = np.round(wl.planted[:, 0] / 0.02) * 0.02
    th0 = np.round(wl.planted[:, 1] / 0.5) * 0.5
    init_l = np.repeat(lam0, 2).astype(np.float32)
    init_t = np.repeat(th0, 2).astype(np.float32)
    out = {}
    with prnu.Context(0) as ctx:
        frames = torch.from_numpy(wl.frames).to(DEV)
        R = torch.empty(frames.shape, device=DEV)
        ctx.prnu_residual(frames, R)
        hs = [ctx.prnu_fingerprint_term(torch.from_numpy(K).to(DEV)) for K in fps]
        t0 = ctx.prnu_get_tuning(H, W)
        try:
            for pers in (0, 2):
                ctx.prnu_set_tuning(H, W, t0["col_width"], t0["pairs_per_block"], t0["wave"], t0["variant"], pers)
                out[pers] = ctx.eis_correction(R, hs, init_l, init_t, max_iter=3, th_half1=20)
        finally:
            ctx.prnu_set_tuning(H, W, t0["col_width"], t0["pairs_per_block"], t0["wave"], t0["variant"],
                                t0["persistent"], t0["streams"], t0["share_forward"])
            for h in hs:
                ctx.prnu_fingerprint_release(h)
    (host, hit), (dev, dit) = out[0], out[2]
    assert np.array_equal(hit, dit)
    for a, b in zip(host.ravel(), dev.ravel()):
        if (a["lam"], a["th_deg"]) == (b["lam"], b["th_deg"]):
            assert (a["dy"], a["dx"], a["cand_idx"]) == (b["dy"], b["dx"], b["cand_idx"])
        assert abs(a["pce"] - b["pce"]) <= 1e-5 * abs(a["pce"])
    # the camera's own fingerprint converges on every frame
    assert np.all(dev[:, 0]["pce"] > 60)
