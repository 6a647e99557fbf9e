"""Host logic of bench.py that the reported numbers rest on (CPU only): the
algorithmic byte model behind the roofline fractions, the clock record that
decides whether a run is kept, and the guard that drops ncu counters taken on
other kernel sources."""
import json
import os
import tempfile

import pytest

import bench


def test_byte_model_per_candidate():
    """1080p FP32: residual 4HW + spectrum 4HW for the row pass, spectrum
    twice plus the fingerprint's half spectrum for the column pass, one
    spectrum read for the row inverse; the kernels add up to the path except
    for the per-row statistics they exchange."""
    H, W = 1080, 1920
    kb = bench.kernel_bytes(H, W, 4, 8)
    assert kb["row_forward"] == 8 * H * W == 16_588_800
    assert kb["column"] == 12 * H * W == 24_883_200
    assert kb["row_inverse"] == 4 * H * W + 16 * H
    assert bench.path_bytes(H, W, 4, 8) == kb["fused"] == 49_766_400
    assert kb["row_forward"] + kb["column"] + kb["row_inverse"] - 16 * H == kb["fused"]
    # FP16 storage: 2-byte residual, 4-byte fingerprint bins
    assert bench.path_bytes(H, W, 2, 4) == 2 * H * W + 36 * H * W // 2 == 41_472_000


def _sampler(lines):
    c = bench.ClockSampler(0)
    fd, c.path = tempfile.mkstemp(suffix=".csv")
    os.close(fd)
    with open(c.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    c.proc = object()
    return c


def test_clock_record_median_and_reasons():
    c = _sampler(["0, 2070, 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active",
                  "0, 2055, 2070, 1400, 0x4, Not Active, Not Active, Not Active, Active",
                  "0, 2070, 2070, 1390, 0x4, Not Active, Not Active, Not Active, Active",
                  "garbage line"])
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert c.summary() == s            # read once, then cached (the sample file is gone)


def test_clock_record_flags_thermal_slowdown():
    c = _sampler(["0, 1500, 2070, 1400, 0x40, Not Active, Active, Not Active, Not Active"])
    assert c.summary()["reasons"] == ["hw_thermal_slowdown"]


def test_counters_are_dropped_when_the_kernel_sources_change(tmp_path, monkeypatch):
    digest = bench.csrc_digest()
    prof = tmp_path / "profiles"
    prof.mkdir()
    entry = {"kernel": "k", "dram_bytes_per_candidate": 1, "warp_instructions_per_candidate": 2}
    (prof / "traffic.json").write_text(json.dumps({
        "column:1080x1920:f32": dict(entry, csrc_digest=digest),
        "row_forward:1080x1920:f32": dict(entry, csrc_digest="0000000000000000"),
    }))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "csrc_digest", lambda: digest)
    assert bench.counters_for("column", 1080, 1920, "f32")["dram_bytes_per_candidate"] == 1
    assert bench.counters_for("row_forward", 1080, 1920, "f32") is None     # taken on other sources
    assert bench.counters_for("column", 2160, 3840, "f16") is None          # never taken


def test_single_process_replica_needs_no_collective():
    r = bench.Replicas("gloo")
    assert (r.ws, r.rank) == (1, 0)
    assert r.max(3.5) == 3.5 and r.whole_job(10, 2.0) == 5.0
    r.barrier()
    r.close()


def test_affinity_ranges_are_compact():
    assert bench._ranges([0, 1, 2, 5, 7, 8]) == "0-2,5,7-8"
    assert bench._ranges([3]) == "3"
    assert bench._ranges([]) == ""


def test_shared_byte_model_reduces_to_the_path_model():
    """With one fingerprint per forward unit the shared byte model charges
    the row pass (s_in HW + 4HW), the forward half in place (8HW) and the
    per-candidate half (read 4HW, fingerprint s_K HW/2, write 4HW) plus the
    row inverse's read (4HW): the path model plus the forward half's extra
    round trip of the spectrum (8HW)."""
    H, W, s_in, s_k = 1080, 1920, 2, 4
    shared = (s_in + 12) * H * W / 1 + (12 + s_k / 2) * H * W
    assert shared == bench.path_bytes(H, W, s_in, s_k) + 8 * H * W


def test_oracle_samples_the_steady_run_else_the_capacity_run():
    assert bench.oracle_sample_queries(16, 100, 20) == list(range(16, 36))
    assert bench.oracle_sample_queries(8, 0, 4) == [0, 1, 2, 3]
    assert bench.oracle_sample_queries(3, 0, 4) == [0, 1, 2]
    assert bench.oracle_sample_queries(16, 5, 20) == list(range(16, 21))
