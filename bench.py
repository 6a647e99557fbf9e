"""Benchmark of the EIS-inversion grid search: warp + xcorr + PCE candidates/s at 1080p.

Workload (default): 30 synthetic stabilised frames of 1920x1080 luma, one
fingerprint, the full 41 x 41 (scale, rotation) grid: 50,430 candidates per
step.  A step is one pass of the whole hot path: noise residual of the 30
frames, fingerprint spectrum, grid search, per-frame arg-max.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is device-timed with the frames already
resident in HBM; `e2e` is the same metric through the C ABI with the frames and
fingerprint in pinned host memory, host<->device copies inside the timed
region.  The reference arm (--impl reference) times the FP64 CPU oracle on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "warp+xcorr+PCE candidates/s at 1080p vs HBM roofline; served p50/p99 query latency"
UNIT = "candidates/s"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--frames", type=int, default=30)
    ap.add_argument("--dtype", choices=["f32", "f16", "bf16"], default="f32")
    ap.add_argument("--no-extras", action="store_true", help="skip the naive-path and CPU-oracle legs")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--workload", choices=["plain", "batched", "precision", "serving", "correction", "literal",
                                                 "denoisers"],
                    default="plain",
                    help="plain = the 1080p metric line; the others print their own JSON record")
    ap.add_argument("--queries", type=int, default=16, help="serving: queries per run")
    ap.add_argument("--wave", type=int, default=0,
                    help="plain workload: candidates per wave after tuning (0 = the tuned value); for small profiles")
    ap.add_argument("--variant", type=int, default=None,
                    help="column-pass variant of the compile-time-planned kernels; -1 = the generic "
                         "runtime-plan kernels (default: the tuned or default variant)")
    ap.add_argument("--autotune-ms", type=float, default=5000.0,
                    help="time budget of the library autotuner run before the warm-up (0 = defaults)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Replicas:
    """One process per GPU, each running its own replica of the workload (the
    search shards by frame and query with no exchange step: weak scaling, no
    collective on the data path).  The only collectives are the timing ones:
    a barrier around the timed region and the maximum of the per-rank times.
    backend "nccl" on GPUs (reductions on `device`), "gloo" on CPU."""

    def __init__(self, backend="nccl", device=None):
        self.ws, self.rank, self.local = dist_env()
        self.backend = backend
        self.device = device
        if self.ws > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)

    def barrier(self):
        if self.ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def max(self, x: float) -> float:
        """The largest x over all ranks (every rank gets it)."""
        if self.ws == 1:
            return float(x)
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device if self.backend == "nccl" else "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def whole_job(self, units_per_rank: int, seconds_per_rank: float) -> float:
        """Units all ranks processed / the slowest rank's time."""
        return units_per_rank * self.ws / self.max(seconds_per_rank)

    def close(self):
        if self.ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


# --------------------------------------------------------------------------- algorithmic bytes

def kernel_bytes(H, W, s_in, s_k):
    """Algorithmic DRAM bytes per candidate of each kernel of the fused path
    (packed half spectrum: H x W/2 complex64 = 4*H*W bytes)."""
    spec = 4 * H * W
    return {
        "row_forward": s_in * H * W + spec,                # read residual, write row spectrum
        "column": spec + s_k * H * W // 2 + spec,          # read, fingerprint spectrum, write
        "row_inverse": spec + 16 * H,                       # read, per-row stats
        "finalize": 16 * H + 12 * 4 * W,                    # stats + the window's rows
        "fused": s_in * H * W + (32 + s_k) * H * W // 2,    # whole path (one pass)
    }


def path_bytes(H, W, s_in, s_k):
    return s_in * H * W + (32 + s_k) * H * (W // 2)


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# the sources that define the planned-plan kernels' device code (and the
# launch shapes chosen for them); host-only files do not change the counters
KERNEL_SOURCES = ("common.cuh", "fft.cuh", "fft_fixed.cuh", "search_common.cuh",
                  "search_fixed.cu", "search_fixed.h", "tma.cuh")


def csrc_digest():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2207_14507_gb300", "csrc")
    for n in KERNEL_SOURCES:
        h.update(n.encode() + open(os.path.join(d, n), "rb").read())
    return h.hexdigest()[:16]


def counters_for(kernel, H, W, dtype):
    """ncu counters per candidate of `kernel` (DRAM bytes, warp instructions)
    from the committed summary profiles/traffic.json, if they were taken on the
    current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    e = d.get(f"{kernel}:{H}x{W}:{dtype}")
    if not e or e.get("csrc_digest") != csrc_digest():
        return None
    return e


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None
        self._summary = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except Exception:
                self.proc.kill()

    def summary(self):
        """Median SM clock, max clock and throttle reasons seen (read once, then cached)."""
        if self._summary is None:
            self._summary = self._read()
        return self._summary or None

    def _read(self):
        if not self.proc or not self.path:
            return {}
        mhz, mx, reasons = [], None, set()
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not mhz:
            return {}
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(mhz)}


# --------------------------------------------------------------------------- CPU oracle leg

def cpu_oracle_sample(wl, target_s, max_cands=200):
    """Time the FP64 oracle, as it stands, on frame 0 of the workload: its
    residual once, then candidates spread over the grid until ~target_s."""
    import oracle
    g = wl.grid
    t0 = time.perf_counter()
    R, _ = oracle.prnu_residual(wl.frames[0])
    K0 = oracle.fingerprint_term(wl.fingerprints[0])
    FK = np.fft.rfft2(K0)
    t_res = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    order = rng.permutation(g.size)
    n = 0
    t1 = time.perf_counter()
    while n < max_cands and (n < 2 or time.perf_counter() - t1 < target_s):
        i, j = divmod(int(order[n]), g.nth)
        oracle.score(R, K0, g.lam_node(i), g.th_node(j), FK)
        n += 1
    t_c = time.perf_counter() - t1
    per_cand = t_c / n + t_res / g.size
    return {"value": 1.0 / per_cand, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"frame 0 of the workload: residual + fingerprint spectrum once, {n} of {g.size} "
                      f"candidates ({t_c:.1f} s), single process, numpy FFT"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import synth
    wl = synth.make_workload(2, F=1)
    H, W = wl.frames.shape[1:]
    per_step = max(1.0, args.cpu_seconds / max(1, args.steps))
    for _ in range(args.warmup):
        cpu_oracle_sample(wl, 0.0, max_cands=1)
    vals = [cpu_oracle_sample(wl, per_step) for _ in range(args.steps)]
    v = statistics.median(x["value"] for x in vals)
    cores = 1
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, H, W, 30),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": vals[0]["sample"]},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args, H, W, F):
    return {"workload": f"plain-1080p: {F} stabilised frames {W}x{H} luma, 1 fingerprint, full 41x41 "
                        f"(scale, rotation) grid, residual + fingerprint spectrum + search per step",
            "frames": F, "H": H, "W": W, "fingerprints": 1, "grid": "41x41",
            "candidates_per_step": F * 1681, "storage": args.dtype,
            "l2": "inputs larger than L2 (frames + residuals 311 MB; >16 GB of spectra streamed per step)"}


# --------------------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    job = Replicas("nccl", dev)

    import synth
    import paper_2207_14507_gb300 as prnu
    prnu.build()

    wl = synth.make_workload(2, F=args.frames)
    F, H, W = wl.frames.shape
    tdt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[args.dtype]
    fpd = {"f32": prnu.PRNU_F32, "f16": prnu.PRNU_F16, "bf16": prnu.PRNU_F16}[args.dtype]
    s_in = 4 if args.dtype == "f32" else 2
    s_k = 8 if args.dtype == "f32" else 4
    flags = prnu.PRNU_WEIGHT_BY_INTENSITY | (0 if args.dtype == "f32" else prnu.PRNU_NORMALISE)
    ncand = F * wl.grid.size

    ctx = prnu.Context(local)
    stream = torch.cuda.current_stream(dev)
    frames_d = torch.from_numpy(wl.frames).to(dev)
    K_d = torch.from_numpy(wl.fingerprints[0]).to(dev)
    R = torch.empty((F, H, W), dtype=tdt, device=dev)
    scale = torch.empty(F, dtype=torch.float32, device=dev)
    out_d = torch.empty((F, 32), dtype=torch.uint8, device=dev)   # prnu_result [F*P]

    tuning = ctx.prnu_autotune(H, W, fpd, budget_ms=args.autotune_ms) if args.autotune_ms > 0 \
        else ctx.prnu_get_tuning(H, W)
    if args.wave > 0 or args.variant is not None:
        tuning = dict(tuning, wave=args.wave if args.wave > 0 else tuning["wave"],
                      variant=args.variant if args.variant is not None else tuning["variant"])
        ctx.prnu_set_tuning(H, W, tuning["col_width"], tuning["pairs_per_block"], tuning["wave"], tuning["variant"],
                            tuning["persistent"])

    def step():
        ctx.prnu_residual(frames_d, R, scale=scale, flags=flags)
        h = ctx.prnu_fingerprint_term(K_d, fpd)
        ctx.eis_grid_search(R, [h], wl.grid, scale=scale, out=out_d)
        ctx.prnu_fingerprint_release(h)

    def barrier():
        job.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = ctx.prnu_launch_count()
    with ClockSampler(local) as clk:
        ctx.prnu_profile_begin()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        barrier()
        prof = ctx.prnu_profile_end()
    launches = ctx.prnu_launch_count() - launches0
    ms = job.max(e0.elapsed_time(e1) / args.steps)
    value = job.whole_job(ncand, ms / 1e3)

    # ---- e2e: the same step through the C ABI from pinned host memory
    frames_h = torch.from_numpy(wl.frames).pin_memory()
    K_h = torch.from_numpy(wl.fingerprints[0]).pin_memory()
    fr2 = torch.empty_like(frames_d)
    K2 = torch.empty_like(K_d)

    def step_e2e():
        fr2.copy_(frames_h, non_blocking=True)
        K2.copy_(K_h, non_blocking=True)
        ctx.prnu_residual(fr2, R, scale=scale, flags=flags)
        h = ctx.prnu_fingerprint_term(K2, fpd)
        res = ctx.eis_grid_search(R, [h], wl.grid, scale=scale)      # host results: D2H + sync inside
        ctx.prnu_fingerprint_release(h)
        return res

    step_e2e()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        res = step_e2e()
    barrier()
    e2e_s = job.max((time.perf_counter() - t0) / args.steps)
    e2e = {"value": job.whole_job(ncand, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": int(wl.frames.nbytes + wl.fingerprints[0].nbytes),
           "d2h_bytes_per_step": int(res.nbytes)}

    # ---- roofline of the dominant kernel (event-timed inside the timed region)
    peak, peak_kind = hbm_peak()
    kb = kernel_bytes(H, W, s_in, s_k)
    timed = {k: v for k, v in prof.items() if k in kb}
    dom = max(timed, key=lambda k: timed[k]["total_ms"])
    cands_total = ncand * args.steps
    achieved = kb[dom] * cands_total / (timed[dom]["total_ms"] / 1e3) / 1e9
    per_launch = cands_total / timed[dom]["launches"]          # candidates one launch of `dom` processes
    cnt = counters_for(dom, H, W, args.dtype)
    traffic = round(cnt["dram_bytes_per_candidate"] * per_launch) if cnt else None
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": f"{peak_kind} hbm_gbs",
            "traffic": traffic, "algorithmic_bytes_per_candidate": kb[dom],
            "candidates_per_launch": round(per_launch, 1),
            "share_of_step": round(timed[dom]["total_ms"] / (ms * args.steps), 3)}
    # The same kernel against the instruction-issue roof: ncu's warp
    # instructions per candidate x candidates/s over 4 issue slots per SM per clock.
    issue = None
    if cnt and cnt.get("warp_instructions_per_candidate"):
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = (clk.summary() or {}).get("sm_mhz") or 2070.0   # median SM clock sampled in the timed region
        slots = nsm * 4 * mhz * 1e6
        rate = cnt["warp_instructions_per_candidate"] * cands_total / (timed[dom]["total_ms"] / 1e3)
        issue = {"bound": "issue", "kernel": dom, "achieved": round(rate / 1e12, 4), "peak": round(slots / 1e12, 4),
                 "unit": "Twarp-inst/s", "frac": round(rate / slots, 4),
                 "warp_instructions_per_candidate": cnt["warp_instructions_per_candidate"]}
    pb = path_bytes(H, W, s_in, s_k)
    path_roof = {"bytes_per_candidate": pb, "achieved": round(pb * value / ws / 1e9, 1),
                 "frac": round(pb * value / ws / 1e9 / peak, 4)}
    kernels = {k: {"launches": v["launches"], "ms_per_step": round(v["total_ms"] / args.steps, 3)}
               for k, v in prof.items()}

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": dict(workload_config(args, H, W, F), tuning=tuning),
        "e2e": e2e, "gpu_launches": int(launches), "roofline": roof, "path_roofline": path_roof,
        "issue_roofline": issue, "kernels": kernels, "clocks": clk.summary(),
    }

    if rank == 0 and not args.no_extras:
        # plain per-candidate GPU path on the same inputs (a sample of frame 0's grid)
        if args.dtype == "f32":
            win = np.array([[18, 22, 18, 22]], np.int32)       # 25 candidates
            Rn = R[:1].contiguous()
            h = ctx.prnu_fingerprint_term(K_d, prnu.PRNU_F32)
            ctx.eis_grid_search(Rn, [h], wl.grid, windows=win, naive=True)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            reps = 4
            for _ in range(reps):
                ctx.eis_grid_search(Rn, [h], wl.grid, windows=win, naive=True)
            torch.cuda.synchronize(dev)
            naive = 25 * reps / (time.perf_counter() - t0)
            ctx.prnu_fingerprint_release(h)
            line["naive_baseline"] = {"value": round(naive, 1), "unit": UNIT,
                                      "speedup": round(value / naive, 2),
                                      "sample": "frame 0, 5x5 window (25 candidates), FP32, one candidate per launch sequence"}
        line["cpu_baseline"] = cpu_oracle_sample(wl, args.cpu_seconds)
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    job.close()


# --------------------------------------------------------------------------- other workloads

def _timed_steps(step, steps, warmup, dev, ctx=None):
    """ms per step over `steps` timed steps after `warmup` untimed ones; with
    `ctx`, also the library's per-kernel profile of the timed steps only."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ctx is not None:
        ctx.prnu_profile_begin()
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize(dev)
    prof = ctx.prnu_profile_end() if ctx is not None else None
    ms = e0.elapsed_time(e1) / steps
    return (ms, prof) if ctx is not None else ms


def run_batched(args):
    """Config 3: 256 full-HD frames in one call, +-k warm-start windows
    (k uniform in 2..10); FP32 (the configuration), or with --dtype f16/bf16
    the FP16-storage variant (residuals with per-frame 1/RMS scale, FP16
    fingerprint spectrum, FP32 arithmetic).  The plain per-candidate FP32
    path runs on a sample of the same inputs for the speedup."""
    import torch
    import synth
    import paper_2207_14507_gb300 as prnu
    prnu.build()
    dev = torch.device("cuda", 0)
    wl = synth.make_workload(3, F=args.frames if args.frames != 30 else 256)
    F, H, W = wl.frames.shape
    win = wl.windows
    ncand = int(sum((w[1] - w[0] + 1) * (w[3] - w[2] + 1) for w in win))
    half = args.dtype != "f32"
    tdt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[args.dtype]
    fpd = prnu.PRNU_F16 if half else prnu.PRNU_F32
    flags = prnu.PRNU_WEIGHT_BY_INTENSITY | (prnu.PRNU_NORMALISE if half else 0)
    s_in, s_k = (2, 4) if half else (4, 8)
    ctx = prnu.Context(0)
    tuning = ctx.prnu_autotune(H, W, fpd, budget_ms=args.autotune_ms) if args.autotune_ms > 0 else None
    frames_d = torch.from_numpy(wl.frames).to(dev)
    K_d = torch.from_numpy(wl.fingerprints[0]).to(dev)
    R = torch.empty((F, H, W), dtype=tdt, device=dev)
    scale = torch.empty(F, device=dev)
    out_d = torch.empty((F, 32), dtype=torch.uint8, device=dev)

    def step():
        ctx.prnu_residual(frames_d, R, scale=scale, flags=flags)
        h = ctx.prnu_fingerprint_term(K_d, fpd)
        ctx.eis_grid_search(R, [h], wl.grid, windows=win, scale=scale, out=out_d)
        ctx.prnu_fingerprint_release(h)

    ms, prof = _timed_steps(step, args.steps, args.warmup, dev, ctx)
    value = ncand / (ms / 1e3)
    res = out_d.cpu().numpy().view(prnu.RESULT_DTYPE).reshape(F)
    hits = int(sum(abs(float(res[f]["lam"]) - wl.planted[f, 0]) <= wl.grid.dlam / 2 + 1e-6 and
                   abs(float(res[f]["th_deg"]) - wl.planted[f, 1]) <= wl.grid.dth_deg / 2 + 1e-6 for f in range(F)))
    # the plain per-candidate FP32 path on the first 4 frames' windows (same inputs)
    R32 = torch.empty((4, H, W), device=dev)
    ctx.prnu_residual(frames_d[:4], R32)
    h = ctx.prnu_fingerprint_term(K_d)
    sub = slice(0, 4)
    nsub = int(sum((w[1] - w[0] + 1) * (w[3] - w[2] + 1) for w in win[sub]))
    ctx.eis_grid_search(R32, [h], wl.grid, windows=win[sub], naive=True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ctx.eis_grid_search(R32, [h], wl.grid, windows=win[sub], naive=True)
    torch.cuda.synchronize(dev)
    naive = nsub / (time.perf_counter() - t0)
    t0 = time.perf_counter()
    ctx.eis_grid_search(R32, [h], wl.grid, windows=win[sub])
    torch.cuda.synchronize(dev)
    fused_sub = nsub / (time.perf_counter() - t0)
    ctx.prnu_fingerprint_release(h)
    peak, kind = hbm_peak()
    pb = path_bytes(H, W, s_in, s_k)
    print(json.dumps({
        "workload": "batched-1080p (config 3)", "metric": "candidates/s", "value": round(value, 1),
        "frames": F, "candidates_per_step": ncand, "window_candidates": [int(((win[1:, 1] - win[1:, 0] + 1) * (win[1:, 3] - win[1:, 2] + 1)).min()),
                              int(((win[1:, 1] - win[1:, 0] + 1) * (win[1:, 3] - win[1:, 2] + 1)).max())],
        "ms_per_step": round(ms, 2), "steps": args.steps, "warmup": args.warmup, "dtype": args.dtype,
        "path_roofline_frac": round(pb * value / 1e9 / peak, 4), "peak": f"{peak} GB/s {kind}",
        "frames_within_half_a_grid_step_of_planted": hits,
        "naive_baseline": {"value": round(naive, 1), "speedup": round(value / naive, 2),
                           "sample": f"first 4 frames' windows ({nsub} candidates), FP32, one call each way",
                           "fused_same_sample_f32": round(fused_sub, 1)},
        "tuning": tuning, "kernels": {k: round(v["total_ms"] / args.steps, 2) for k, v in prof.items()},
    }), flush=True)
    ctx.close()


def run_correction(args):
    """The iterative correction of Sec. 3.2 (eis_correction) on full-HD frames
    with continuous planted transforms, started from a coarse estimate: 3
    iterations at most, the text's dense first angle grid (11 scales x 101
    angles, then 11 x 11 twice).  Reports
    frames/s and candidates/s (nodes scored), the iterations used, and the FP64
    oracle's candidates/s on a bounded sample of the first iteration's nodes."""
    import torch
    import oracle
    import synth
    import paper_2207_14507_gb300 as prnu
    prnu.build()
    dev = torch.device("cuda", 0)
    F = args.frames if args.frames != 30 else 8
    wl = synth.make_workload(2, F=F)
    F, H, W = wl.frames.shape
    ctx = prnu.Context(0)
    tuning = ctx.prnu_autotune(H, W, prnu.PRNU_F32, budget_ms=args.autotune_ms) if args.autotune_ms > 0 else None
    frames_d = torch.from_numpy(wl.frames).to(dev)
    K_d = torch.from_numpy(wl.fingerprints[0]).to(dev)
    R = torch.empty((F, H, W), device=dev)
    ctx.prnu_residual(frames_d, R)
    h = ctx.prnu_fingerprint_term(K_d)
    state = {}
    # start estimates: the planted transform snapped to a coarse lattice (0.02
    # in scale, 0.5 degree), standing in for the paper's initialisation from
    # the SIFT co-registration of consecutive frames
    init_l = (np.round(wl.planted[:, 0] / 0.02) * 0.02).astype(np.float32)
    init_t = (np.round(wl.planted[:, 1] / 0.5) * 0.5).astype(np.float32)

    def step():
        state["out"], state["its"] = ctx.eis_correction(R, [h], init_lam=init_l, init_th=init_t, max_iter=3,
                                                        th_half1=50)

    ms = _timed_steps(step, args.steps, max(args.warmup, 1), dev)
    its = state["its"][:, 0]
    nodes = int(sum(11 * 101 + 121 * (int(k) - 1) for k in its))
    out = state["out"][:, 0]
    err_l = float(np.max(np.abs(out["lam"] - wl.planted[:, 0])))
    err_t = float(np.max(np.abs(out["th_deg"] - wl.planted[:, 1])))
    # the oracle on a bounded sample of the first iteration's nodes of frame 0
    t0 = time.perf_counter()
    Rh = oracle.prnu_residual(wl.frames[0])[0]
    K0 = oracle.fingerprint_term(wl.fingerprints[0])
    FK = np.fft.rfft2(K0)
    lams, ths = oracle.correction_nodes(1.0, 0.0, 1)
    n = 0
    t1 = time.perf_counter()
    while n < 200 and (n < 2 or time.perf_counter() - t1 < args.cpu_seconds):
        oracle.score(Rh, K0, lams[n % 11], ths[(7 * n) % 101], FK)
        n += 1
    t_c = time.perf_counter() - t1
    cpu = {"value": round(n / t_c, 3), "unit": "candidates/s", "cores": 1, "kind": "oracle",
           "sample": f"frame 0: {n} first-iteration nodes ({t_c:.1f} s, residual {t1 - t0:.1f} s apart), "
                     f"single process, numpy FFT"}
    peak, kind = hbm_peak()
    print(json.dumps({
        "workload": "correction-1080p (Sec. 3.2 iterative search)", "metric": "frames/s",
        "value": round(F / (ms / 1e3), 3), "frames": F, "ms_per_step": round(ms, 2), "steps": args.steps,
        "candidates_per_s": round(nodes / (ms / 1e3), 1), "nodes_per_step": nodes,
        "iterations": [int(k) for k in its], "max_abs_error_vs_planted": {"lam": err_l, "th_deg": err_t},
        "path_roofline_frac": round(path_bytes(H, W, 4, 8) * nodes / (ms / 1e3) / 1e9 / peak, 4),
        "peak": f"{peak} GB/s {kind}", "tuning": tuning, "cpu_baseline": cpu, "dtype": "f32",
    }), flush=True)
    ctx.close()


def run_literal(args):
    """The frame-literal search of Sec. 3.2 (eis_grid_search_frames: warp the
    frame and extract the residual for every candidate) on the full-HD
    workload, 4 frames x 1681 candidates by default.  Reports candidates/s,
    the per-kernel split, the path roofline of the byte model plus the render
    (two passes over the uint8 frame and the FP32 residual written: 6 HW bytes
    per candidate), the same frames through eis_grid_search (residual once
    per frame) for comparison, and the FP64 oracle on a bounded sample."""
    import torch
    import oracle
    import synth
    import paper_2207_14507_gb300 as prnu
    prnu.build()
    dev = torch.device("cuda", 0)
    F = args.frames if args.frames != 30 else 4
    wl = synth.make_workload(2, F=F)
    F, H, W = wl.frames.shape
    ncand = F * wl.grid.size
    ctx = prnu.Context(0)
    tuning = ctx.prnu_autotune(H, W, prnu.PRNU_F32, budget_ms=args.autotune_ms) if args.autotune_ms > 0 else None
    frames_d = torch.from_numpy(wl.frames).to(dev)
    K_d = torch.from_numpy(wl.fingerprints[0]).to(dev)
    h = ctx.prnu_fingerprint_term(K_d)
    state = {}

    def step():
        state["r"] = ctx.eis_grid_search_frames(frames_d, [h], wl.grid)

    ms, prof = _timed_steps(step, args.steps, max(args.warmup, 1), dev, ctx)
    R = torch.empty((F, H, W), device=dev)

    def step_resid():
        ctx.prnu_residual(frames_d, R)
        state["q"] = ctx.eis_grid_search(R, [h], wl.grid)

    ms_r = _timed_steps(step_resid, args.steps, max(args.warmup, 1), dev)
    got = state["r"][:, 0]
    # the oracle on a bounded sample: literal candidates of frame 0
    K0 = oracle.fingerprint_term(wl.fingerprints[0])
    FK = np.fft.rfft2(K0)
    cands = oracle.candidate_list(wl.grid)
    n, t1 = 0, time.perf_counter()
    while n < 200 and (n < 2 or time.perf_counter() - t1 < args.cpu_seconds):
        idx, lam, th = cands[(37 * n) % len(cands)]
        oracle.score_literal(wl.frames[0], K0, lam, th, True, FK)
        n += 1
    t_c = time.perf_counter() - t1
    cpu = {"value": round(n / t_c, 3), "unit": "candidates/s", "cores": 1, "kind": "oracle",
           "sample": f"frame 0: {n} literal candidates ({t_c:.1f} s), single process, numpy FFT"}
    peak, kind = hbm_peak()
    value = ncand / (ms / 1e3)
    planted_hits = int(sum(abs(float(got[f]["lam"]) - wl.planted[f, 0]) <= 0.0025 + 1e-6 and
                           abs(float(got[f]["th_deg"]) - wl.planted[f, 1]) <= 0.125 + 1e-6 for f in range(F)))
    print(json.dumps({
        "workload": "literal-1080p (Sec. 3.2: frame warped and residual extracted per candidate)",
        "metric": "candidates/s", "value": round(value, 1), "unit": "candidates/s", "frames": F,
        "candidates_per_step": ncand, "ms_per_step": round(ms, 2), "steps": args.steps, "dtype": "f32",
        "path_roofline_frac": round((path_bytes(H, W, 4, 8) + 6 * H * W) * value / 1e9 / peak, 4),
        "residual_once_per_frame": {"value": round(ncand / (ms_r / 1e3), 1), "ms_per_step": round(ms_r, 2)},
        "frames_within_half_a_grid_step_of_planted": planted_hits,
        "kernels": {k: round(v["total_ms"] / args.steps, 2) for k, v in prof.items()},
        "peak": f"{peak} GB/s {kind}", "tuning": tuning, "cpu_baseline": cpu,
    }), flush=True)
    ctx.close()


def run_denoisers(args):
    """The two residual extractors on the full-HD workload's 30 frames: the 3x3
    Wiener filter (prnu_residual) and Mihcak's wavelet denoiser
    (prnu_residual_wavelet, sigma0 = 3), FP32 output.  Reports frames/s of
    each, the Wiener kernel's HBM fraction (one uint8 read and one FP32
    write per pixel), and the FP64 oracle's frames/s for each on one core."""
    import torch
    import oracle
    import synth
    import paper_2207_14507_gb300 as prnu
    prnu.build()
    dev = torch.device("cuda", 0)
    wl = synth.make_workload(2, F=args.frames)
    F, H, W = wl.frames.shape
    ctx = prnu.Context(0)
    frames_d = torch.from_numpy(wl.frames).to(dev)
    R = torch.empty((F, H, W), device=dev)
    ms_w = _timed_steps(lambda: ctx.prnu_residual(frames_d, R), args.steps, max(args.warmup, 3), dev)
    ms_v = _timed_steps(lambda: ctx.prnu_residual_wavelet(frames_d, R, 3.0), args.steps, max(args.warmup, 3), dev)
    t0 = time.perf_counter()
    oracle.prnu_residual(wl.frames[0])
    t1 = time.perf_counter()
    oracle.prnu_residual_wavelet(wl.frames[0], 3.0)
    t2 = time.perf_counter()
    peak, kind = hbm_peak()
    print(json.dumps({
        "workload": "denoisers-1080p (Sec. 2.2 residual: 3x3 Wiener and Mihcak wavelet)", "metric": "frames/s",
        "frames": F, "steps": args.steps, "dtype": "f32",
        "wiener": {"value": round(F / (ms_w / 1e3), 1), "ms_per_step": round(ms_w, 3),
                   "hbm_frac": round(5 * H * W * F / (ms_w / 1e3) / 1e9 / peak, 4)},
        "wavelet": {"value": round(F / (ms_v / 1e3), 1), "ms_per_step": round(ms_v, 3)},
        "cpu_baseline": {"unit": "frames/s", "cores": 1, "kind": "oracle", "sample": "frame 0, one each",
                         "wiener": round(1 / (t1 - t0), 3), "wavelet": round(1 / (t2 - t1), 3)},
        "peak": f"{peak} GB/s {kind}",
    }), flush=True)
    ctx.close()


def run_precision(args):
    """Config 4: 32 frames of 3840x2160, full 41x41 grid, half of the frames
    from an independent fingerprint; FP16 and BF16 residual storage with an
    FP16 fingerprint spectrum (FP32 arithmetic), and FP32 for comparison."""
    import torch
    import synth
    import paper_2207_14507_gb300 as prnu
    prnu.build()
    dev = torch.device("cuda", 0)
    wl = synth.make_workload(4, F=args.frames if args.frames != 30 else 32)
    F, H, W = wl.frames.shape
    ncand = F * wl.grid.size
    ctx = prnu.Context(0)
    frames_d = torch.from_numpy(wl.frames).to(dev)
    K_d = torch.from_numpy(wl.fingerprints[0]).to(dev)
    peak, kind = hbm_peak()
    legs = {}
    for name, tdt, fpd, s_in, s_k, flags in (
            ("f16", torch.float16, prnu.PRNU_F16, 2, 4, prnu.PRNU_WEIGHT_BY_INTENSITY | prnu.PRNU_NORMALISE),
            ("bf16", torch.bfloat16, prnu.PRNU_F16, 2, 4, prnu.PRNU_WEIGHT_BY_INTENSITY | prnu.PRNU_NORMALISE),
            ("f32", torch.float32, prnu.PRNU_F32, 4, 8, prnu.PRNU_WEIGHT_BY_INTENSITY)):
        tuning = ctx.prnu_autotune(H, W, fpd, budget_ms=args.autotune_ms) if args.autotune_ms > 0 else None
        R = torch.empty((F, H, W), dtype=tdt, device=dev)
        scale = torch.empty(F, device=dev)
        res = {}

        def step():
            ctx.prnu_residual(frames_d, R, scale=scale, flags=flags)
            h = ctx.prnu_fingerprint_term(K_d, fpd)
            res["r"] = ctx.eis_grid_search(R, [h], wl.grid, scale=scale)
            ctx.prnu_fingerprint_release(h)

        ms, prof = _timed_steps(step, args.steps, args.warmup, dev, ctx)
        value = ncand / (ms / 1e3)
        pce = res["r"]["pce"][:, 0]
        legs[name] = {"value": round(value, 1), "ms_per_step": round(ms, 1),
                      "path_roofline_frac": round(path_bytes(H, W, s_in, s_k) * value / 1e9 / peak, 4),
                      "matched_min_pce": float(pce[wl.frame_fp == 0].min()) if (wl.frame_fp == 0).any() else None,
                      "unmatched_max_pce": float(pce[wl.frame_fp == 1].max()) if (wl.frame_fp == 1).any() else None,
                      "decisions_at_60": [bool(p >= 60) for p in pce], "tuning": tuning,
                      "kernels": {k: round(v["total_ms"] / args.steps, 1) for k, v in prof.items()}}
    print(json.dumps({"workload": "precision-4k (config 4)", "metric": "candidates/s", "frames": F,
                      "candidates_per_step": ncand, "steps": args.steps, "warmup": args.warmup,
                      "peak": f"{peak} GB/s {kind}", "legs": legs}), flush=True)
    ctx.close()


def run_serving(args):
    """Config 5: Poisson query stream (720p/1080p/4K, 8-64 frames, 1-16
    fingerprints, one matching with probability 0.5, +-k windows, FP16
    storage, 120 GB admission budget).  Three runs: all queries at once
    (capacity), a Poisson stream at 70% of the measured capacity, and the
    nominal 20 queries/s (overloaded)."""
    import threading
    import torch
    import synth
    import paper_2207_14507_gb300 as prnu
    prnu.build()
    dev = torch.device("cuda", 0)
    n = args.queries
    queries, banks = synth.make_query_stream(3 * n, rate_hz=20.0, pool_frames=8, match_sources=1)
    ctx = prnu.Context(0, hbm_budget_bytes=120 << 30)
    tunings = {}
    for (H, W) in banks:
        tunings[f"{H}x{W}"] = ctx.prnu_autotune(H, W, prnu.PRNU_F16, budget_ms=args.autotune_ms) \
            if args.autotune_ms > 0 else None
    handles = {k: [ctx.prnu_fingerprint_term(torch.from_numpy(K).to(dev), prnu.PRNU_F16) for K in bank]
               for k, bank in banks.items()}
    frames = [torch.from_numpy(q.frames).to(dev) for q in queries]
    torch.cuda.synchronize(dev)
    ncand = [len(q.fp_ids) * int(sum((w[1] - w[0] + 1) * (w[3] - w[2] + 1) for w in q.windows)) for q in queries]

    def submit(q, fr):
        hs = [handles[(q.H, q.W)][i] for i in q.fp_ids]
        return ctx.query_submit(fr, hs, synth.GRID_FULL, windows=q.windows, dtype=prnu.PRNU_F16,
                                flags=prnu.PRNU_WEIGHT_BY_INTENSITY | prnu.PRNU_NORMALISE)

    def run(idx, arrivals):
        ids = {}
        done = []

        def poller():
            for i in idx:
                while i not in ids:
                    time.sleep(0.0005)
                ctx.query_poll(ids[i], queries[i].frames.shape[0], len(queries[i].fp_ids), timeout_us=-1)
                done.append(i)

        th = threading.Thread(target=poller)
        th.start()
        t0 = time.perf_counter()
        for i, t in zip(idx, arrivals):
            now = time.perf_counter() - t0
            if t > now:
                time.sleep(t - now)
            ids[i] = submit(queries[i], frames[i])
        th.join()
        wall = time.perf_counter() - t0
        lat = np.array([ctx.query_latency(ids[i])["total_ms"] for i in idx])
        return wall, lat

    # capacity: everything at once
    idx0 = list(range(0, n))
    wall, lat = run(idx0, [0.0] * n)
    cap_q = n / wall
    cap_c = sum(ncand[i] for i in idx0) / wall
    # Poisson at 70% of capacity, and at the nominal 20 queries/s
    rng = np.random.default_rng(5)
    out = {}
    for name, rate, idx in (("70pct_capacity", 0.7 * cap_q, list(range(n, 2 * n))),
                            ("20qps_overloaded", 20.0, list(range(2 * n, 3 * n)))):
        arr = np.cumsum(rng.exponential(1.0 / rate, size=len(idx)))
        w2, l2 = run(idx, list(arr))
        out[name] = {"rate_qps": round(rate, 3), "queries": len(idx), "wall_s": round(w2, 2),
                     "throughput_qps": round(len(idx) / w2, 3),
                     "candidates_per_s": round(sum(ncand[i] for i in idx) / w2, 1),
                     "p50_ms": round(float(np.percentile(l2, 50)), 1), "p99_ms": round(float(np.percentile(l2, 99)), 1),
                     "overloaded": bool(rate > cap_q)}
    st = ctx.prnu_server_stats_get()
    print(json.dumps({"workload": "serving (config 5)", "metric": "served p50/p99 query latency",
                      "capacity": {"queries_per_s": round(cap_q, 3), "candidates_per_s": round(cap_c, 1),
                                   "queries": n, "p50_ms": round(float(np.percentile(lat, 50)), 1),
                                   "p99_ms": round(float(np.percentile(lat, 99)), 1)},
                      "runs": out, "mean_candidates_per_query": round(float(np.mean(ncand)), 1),
                      "budget_gb": 120, "admitted_bytes_peak": st["admitted_bytes_peak"],
                      "server_launches": st["server_launches"], "dtype": "f16", "tuning": tunings}), flush=True)
    ctx.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "precision":
        run_precision(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "correction":
        run_correction(args)
    elif args.workload == "literal":
        run_literal(args)
    elif args.workload == "denoisers":
        run_denoisers(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
