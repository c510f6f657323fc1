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


def test_oracle_many_equals_one_by_one():
    import oracle

    specs = [synth.small_spec(60 + k, 96 + 16 * k, 64, n=3, levels=3, ref=1) for k in range(4)]
    stacks = [synth.make_stack(sp).numpy() for sp in specs]
    jobs = [(lambda k=k: (stacks[k], specs[k].levels, specs[k].noise_tol, specs[k].ref)) for k in range(4)]
    many = bench.oracle_many(jobs, 3)
    for k, r in enumerate(many):
        one = oracle.align_stack(stacks[k], specs[k].levels, specs[k].noise_tol, specs[k].ref)
        for key in ("shifts", "level_errs", "level_shifts"):
            assert np.array_equal(r[key], one[key]), (k, key)


def test_reference_arm_times_whole_stacks(capsys):
    import json

    bench.main(["--impl", "reference", "--workload", "pair640x480", "--steps", "2", "--warmup", "1"])
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["config"]["workload"] == "pair640x480"
    assert line["unit"] == "MPix/s" and line["value"] > 0 and line["e2e"]["value"] == line["value"]
    assert "whole pair640x480 stack" in line["cpu_baseline"]["sample"]
