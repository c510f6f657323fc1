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


def test_serve_summary_keeps_the_checked_counts():
    """The served run folded into the default line keeps, per offered rate,
    the latency and both equality counts, and relates the best served rate to
    the plain path on the same jobs."""
    rates = [{"offered_jobs_s": r, "jobs": 64, "served_jobs_s": min(r, 400.0), "mpix_s": 144.0 * min(r, 400.0),
              "p50_ms": 2.7, "p99_ms": 5.0, "same_as_alone": "64/64", "oracle_equal": "64/64",
              "queue_p50_ms": 0.01, "h2d_gbs": 1.0} for r in (10.0, 100.0, 1000.0)]
    line = {"value": 57600.0, "unit": "MPix/s",
            "config": {"workload": "serve6000x4000x7", "pool_jobs": 8, "slots": 8, "budget_gb": 40.0},
            "plain_path_device_resident": {"mpix_s": 576000.0}, "roofline": {"frac": 0.97}, "serving": rates,
            "alone_equal_oracle": "8/8", "oracle_check": "every served job", "server_stats": {"failed": 0}}
    s = bench.serve_summary(line)
    assert s["value"] == 57600.0 and s["served_vs_plain"] == 0.1 and s["h2d_link_frac"] == 0.97
    assert [r["offered_jobs_s"] for r in s["rates"]] == [10.0, 100.0, 1000.0]
    assert all(r["oracle_equal"] == "64/64" and r["same_as_alone"] == "64/64" for r in s["rates"])
    assert "queue_p50_ms" not in s["rates"][0]
    assert s["alone_equal_oracle"] == "8/8" and s["server_stats"]["failed"] == 0


def test_default_line_folds_in_a_short_served_run():
    args = bench.parse_args([])
    assert args.workload == "stack6000x4000x7" and args.serve_pool > 0 and args.batch_count == 256
    assert args.min_timed_s >= 0.5
