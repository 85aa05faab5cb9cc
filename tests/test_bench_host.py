"""Host-side pieces of bench.py that need no GPU: the bounded CPU-oracle
sample behind cpu_baseline and the reference arm, the clock sampler's
behaviour without nvidia-smi readings, the committed profile's traffic
record, and the whole-job arithmetic."""
import os
import re

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_cpu_oracle_sample_is_bounded_and_positive():
    from oracle import build as obuild
    obuild.build()
    v, n, t = bench.cpu_oracle_sample(target_s=0.3)
    assert v > 0 and n >= 1024 and t > 0
    assert abs(v - n * bench.D / t) <= 1e-6 * v
    # the sample is sized from a probe: it should land near the target, not
    # at the 131072-row cap
    assert n < bench.D


def test_clock_sampler_without_readings():
    c = bench.ClockSampler(0)
    c.proc = None  # as when nvidia-smi is absent
    out = c.stop()
    assert out["samples"] == 0 and out["sm_mhz"] is None and out["reasons"] == []


def test_profile_traffic_record_parses():
    """The dominant kernel's summary carries a per-launch DRAM figure and the
    hash of the source it was taken on; bench.py reports the figure only
    while the hash matches."""
    txt = open(os.path.join(ROOT, "profiles", "dvr_rows_f32_D131072.md")).read()
    assert re.search(r"traffic_bytes_per_launch:\s*[0-9.eE+]+", txt)
    assert re.search(r"source_sha256:\s*[0-9a-f]{64}", txt)
    t = bench.traffic_from_profile()
    assert t is None or 1e5 < t < 1e8


@pytest.mark.parametrize("world", [1, 2, 8])
def test_job_value_is_whole_job_throughput(world):
    assert bench.job_value(world, 10, 1e9, 2.0) == pytest.approx(world * 10 * 1e9 / 2.0)


def test_per_pipe_bound_takes_the_slowest_pipe():
    """The generation roofline: each pipe's operations per canonical entry
    over its rate; the bound is the slowest pipe, the sum the no-overlap
    bound, and a kernel at exactly the bound's rate has frac 1."""
    rates = {"imad_hi": 1e13, "imad": 2e13, "lop3": 2e13, "iadd3": 2e13, "ffma": 4e13, "mufu": 5e12, "i2f": 5e12}
    b = bench.pipe_bound(rates)
    ops = b["ops_per_entry"]
    assert ops["ffma"] == bench.PHILOX_GEN_PIPE_OPS["ffma"] + 8
    assert sum(bench.PHILOX_GEN_PIPE_OPS.values()) == 103  # 39 integer Philox ops + the rest of the definition
    t = {k: ops[k] / rates[k] for k in ops}
    assert b["bound_pipe"] == max(t, key=t.get) and b["t_bound"] == max(t.values())
    assert abs(b["t_sum"] - sum(t.values())) < 1e-30
    r = bench.pipe_roofline(1.0 / b["t_bound"], rates)
    assert abs(r["frac"] - 1.0) < 1e-12 and r["sum_frac"] > 1.0
    assert bench.pipe_bound(rates, apply_ffma_per_entry=0)["ops_per_entry"]["ffma"] == 46


def test_fp64_roofline_counts_the_definition():
    """The FP64 form's bound: 51 FP64 operations of the definition per
    canonical entry (two uniforms, log with its division and polynomial,
    square root, sin/cos polynomials, scaling) plus 8 apply FMAs, over the
    measured DFMA rate; without rates no fraction is claimed."""
    assert bench.PHILOX64_DFMA_OPS == 51
    r = bench.fp64_roofline(1e6, 1e-3, {"dfma": 5.9e10})
    assert r["ops_per_entry"] == 59 and abs(r["frac"] - 1.0) < 1e-12
    assert "frac" not in bench.fp64_roofline(1e6, 1e-3, None)


def test_batch_roofline_reports_the_pairs_once_bound():
    """The batched roofline takes the stored bytes the chosen forms read and,
    beside it, the bound with every stored pair read once (half the
    row-owner bytes)."""
    import bench
    r = bench.batch_roofline(8e9, 0.0, 1e9, 2e-3, None, 4e9)
    hbm = bench.measured_peaks()["hbm_gbs"] * 1e9
    assert abs(r["t_hbm_s"] - 8e9 / hbm) < 1e-12 and abs(r["t_hbm_pairs_once_s"] - 4e9 / hbm) < 1e-12
    assert r["bound"] == "hbm" and abs(r["frac"] - (8e9 / hbm) / 2e-3) < 1e-9
    assert abs(r["frac_of_pairs_once_bound"] - max(4e9 / hbm, r["t_fma_s"]) / 2e-3) < 1e-9
    assert "t_hbm_pairs_once_s" not in bench.batch_roofline(8e9, 0.0, 1e9, 2e-3)
