"""Host-side parts of bench.py that need no GPU: the percentile used for the
latency figures, the host description recorded with the oracle baselines, and
the threaded oracle baseline on a small stack."""
import os

import numpy as np

import bench
from paper_2007_06483_gb300 import synth


def test_percentile_is_nearest_rank():
    xs = list(range(1, 101))
    assert bench._pct(xs, 0.50) == 50
    assert bench._pct(xs, 0.99) == 99
    assert bench._pct(xs, 1.00) == 100
    assert bench._pct([7.0], 0.99) == 7.0
    assert bench._pct([3, 1, 2], 0.5) == 2  # order of the samples does not matter


def test_latency_loop_meets_the_sample_rule():
    assert bench.LAT_STEPS >= 100 and bench.LAT_WARMUP >= 10


def test_host_cpu_record():
    h = bench.host_cpu()
    assert h["nproc"] == os.cpu_count()
    assert 1 <= h["usable_cores"] <= h["nproc"]
    assert isinstance(h["arch"], str) and h["arch"]
    assert h["model"] is None or isinstance(h["model"], str)


def test_threaded_oracle_baseline_small_stack():
    spec = bench.workload("pair640x480")
    images = synth.make_stack(spec).numpy()
    single = bench.oracle_rate(images, spec, budget_s=0.3)
    assert np.array_equal(single["result"]["shifts"], synth.expected_shifts(spec))
    r = bench.oracle_rate_threaded(images, spec, 2, budget_s=0.3)
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["value"] > 0
    assert "2 threads" in r["sample"]
