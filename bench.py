#!/usr/bin/env python3
"""Benchmark of the MTB alignment hot path on one or more GB300s.

A step is one pass of the whole path over one exposure stack: one
mtb_align_stack_ex call, which enqueues the pyramid pass (k_clear, k_pyramid),
the bitmap pass (k_bitmaps) and the coarse-to-fine shift search (the item
kernel k_search_items, which starts while the bitmaps are still being packed),
chained by programmatic dependent launch.  The stage split times the search
on its own, where the library picks the staged kernel (k_search_staged) for
large stacks.  The
default workload is the 6000x4000 stack of 7 exposures (6 pairs, 8 levels), the
largest plain stack.  The metric is aligned MPix/s: full-resolution pixels of
every aligned pair divided by the step time.  The K timed steps run back to
back between two events: an event between two steps would serialise one step's
search with the next step's launches.  That K-step region is timed again and
again (each time bracketed by a barrier and a synchronize) until the regions
add up to at least --min-timed-s of wall time, so that the clock sampler sees
the GPU under load; the value is the mean over all of them. p50/p99 latency
comes from a second loop with events around each step (at least 100 timed
steps after 10 more warm-ups). A third loop times the same work through the
three stage calls (mtb_build_pyramids, mtb_build_bitmaps, mtb_search_shifts)
with CUDA events between them on the launching stream: the split by stage.  The
roofline names the stage with the largest share of that split, and every
stage's fraction of the peak is listed.

The default line also carries a compact batched-vs-plain record (`batch`): the
uneven stacks of the batched form (--batch-count of them, 256 by default) in
one persistent launch against the plain path on the same stacks, with every
stack's shifts and per-level errors compared with the oracle (run on every
usable host core, outside the timed regions), and a compact served record
(`serve`): a short run of the serving loop (--serve-pool distinct 6000x4000x7
jobs, 64 Poisson arrivals at each of 10, 100 and 1000 jobs/s offered) with
p50/p99 latency per rate, the served MPix/s against the plain path on the same
jobs, and every served job's shifts compared with the oracle's.

Inputs and workspaces rotate over several device copies, so between two uses of
one buffer more than 3x the L2 capacity is written and read: every step starts
with its data in HBM.  `e2e` times the host-buffer entry point
(mtb_align_stack_host) from pinned host memory: copy in, align, copy the shifts
out.  `cpu_baseline` times the single-threaded oracle on the same stack;
`cpu_baseline_threaded` runs that oracle on every usable host core at once,
each thread aligning whole stacks (labelled with the thread count).

Other workloads: `batchN` (N uneven stacks in one persistent launch, against the
plain path), `serve` (Poisson arrivals of 6000x4000x7 jobs into the serving
loop under a 40 GB budget, swept over offered load; p50/p99 latency and served
MPix/s per rate), `apply` (moving the 6000x4000x7 exposures by their shifts)
and `paper` (2560x1440 stacks of 2..7 exposures end to end, with the chain
mode, the quadrant test and the shift application beside).

Multi-GPU (torchrun): each rank aligns its own stack every step (weak scaling,
no collective on the data path); the barrier and the max over ranks of the
timed region are the only cross-rank operations.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "aligned MPix/s per exposure pair"
UNIT = "MPix/s"
# plain-path latency: p50/p99 over at least LAT_STEPS timed steps after
# LAT_WARMUP untimed ones
LAT_STEPS = 100
LAT_WARMUP = 10
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
L2_BYTES = 126 * 1024 * 1024  # GB300 L2 capacity

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture, keyed by kernel and workload, with the SHA-256 of that kernel's
# sources at capture time; reported only while those sources are unchanged.
NCU_TRAFFIC = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum (cold cache), per
    # launch: k_pyramid of the 4000x3000x3 stack (109.70 MB read + 6.95 MB
    # written) and k_apply_shifts of the 6000x4000x7 stack (496.81 + 458.26 MB)
    ("k_pyramid", "stack4000x3000x3"): {"bytes": 116647680, "sources_sha256": "51d50f00dfb4fe6bf0b3fbd829edfbd37d05433985f0057cd6a55eace28f9b84"},
    ("k_apply_shifts", "apply6000x4000x7"): {"bytes": 955071744, "sources_sha256": "e265c02bbfa6e0cda0bd4c35ae4a6118438da478c9b3a3a35471b1d9ce84ba18"},
    # the 6000x4000x7 stack, `bench.py --profile --steps 2 --warmup 2` under
    # ncu, mean over the captured launches: k_pyramid 531.86 MB read + 168.06 MB
    # written (4 launches), k_bitmaps 224.73 + 5.79 MB (4), k_search_staged
    # 56.38 + 0.00 MB (2), k_search_items 56.33 + 0.00 MB (2). Written bytes
    # still dirty in L2 when a launch ends are not counted, hence writes below
    # the algorithmic figure
    ("k_pyramid", "stack6000x4000x7"): {"bytes": 699921664, "sources_sha256": "05c99d248177ca13fecc586c0b584e768a7905956a261b2f4019a54686f47c17"},
    ("k_bitmaps", "stack6000x4000x7"): {"bytes": 230528832, "sources_sha256": "93c617e24e66bcec772aa1f012ed0bed6cfdfd28c5bd3fd6a1d5a04c15920634"},
    ("k_search_staged", "stack6000x4000x7"): {"bytes": 56384640, "sources_sha256": "370439610f1f1c12706f9c510e9d8b31872879be9448a85d34844dc31c9adb56"},
    ("k_search_items", "stack6000x4000x7"): {"bytes": 56329856, "sources_sha256": "178915f00529fb7ac0a627038292eda2fcefa5a468a415e9cfbd054a949c4dac"},
}


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=("gb300", "reference"), default="gb300")
    p.add_argument("--workload", default="stack6000x4000x7")
    p.add_argument("--min-timed-s", type=float, default=5.0,
                   help="repeat the K-step timed region until the regions add up to this many seconds")
    p.add_argument("--batch-count", type=int, default=256,
                   help="stacks of the batched-vs-plain record in the default line (0: leave it out)")
    p.add_argument("--profile-steps", type=int, default=0,
                   help="only run this many plain steps of the workload (for ncu captures) and exit")
    p.add_argument("--buffers", type=int, default=4, help="device copies rotated over the steps")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--profile", action="store_true",
                   help="only the kernels, for ncu: W one-call steps, then K one-call steps and K stage-split steps "
                        "of the plain workload; prints one line of shifts")
    p.add_argument("--cpu-threads", type=int, default=0,
                   help="threads of the threaded oracle baseline (0: the usable cores; 1: skip it)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--rates", default="10,30,100,300,1000,2000", help="serve: offered jobs/s")
    p.add_argument("--pool", type=int, default=32, help="serve: distinct pre-generated jobs")
    p.add_argument("--slots", type=int, default=8, help="serve: jobs on the GPU at most")
    p.add_argument("--copy-streams", type=int, default=1, help="serve: copy streams per job")
    p.add_argument("--budget-gb", type=float, default=40.0, help="serve: device-memory budget")
    p.add_argument("--serve-pool", type=int, default=8,
                   help="default workload: jobs of the short served run folded into the line (0: none)")
    return p.parse_args(argv)


# ----------------------------------------------------------------------------- distributed
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def shard_units(total_units: int, rank: int, world: int):
    """Units (stacks) of one step given to `rank`: contiguous, balanced."""
    lo = total_units * rank // world
    hi = total_units * (rank + 1) // world
    return list(range(lo, hi))


def max_over_ranks(value: float, world: int, device=None) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ----------------------------------------------------------------------------- workload
def workload(name: str):
    from paper_2007_06483_gb300 import synth

    for spec in synth.PLAIN_CONFIGS:
        if spec.name == name:
            return spec
    raise SystemExit(f"unknown workload {name}; choose from {[s.name for s in synth.PLAIN_CONFIGS]}")


def plain_config(spec, world: int, buffers: int) -> dict:
    """The `config` of a plain-stack line, the same for the GPU arm and the
    reference arm (which aligns the same stack on the host cores)."""
    return {"workload": spec.name, "w": spec.w, "h": spec.h, "n_exposures": spec.n, "pairs": spec.pairs,
            "levels": spec.levels, "noise_tol": spec.noise_tol, "ref": spec.ref,
            "stacks_per_step_per_gpu": 1, "parallelism": f"replicas x{world}",
            "l2": f"inputs+workspaces rotate over {buffers} device copies"
                  + (" (the inputs alone > 3x L2)" if buffers * spec.input_bytes > 3 * L2_BYTES
                     else " (they fit in L2: steps may hit it)")}


def algorithmic_bytes(spec) -> dict:
    """Bytes each stage must move for one stack (per step), by the path's design:
    pyramid: read RGB (3 B/px) + write gray of levels 0..min(L-1, 5);
    bitmaps: read every gray level (1 B/px) + write tb and eb (2 bits/px), plus
             the deep levels' own gray writes;
    search:  read tb and eb of both exposures at every level (4 bits/px/pair)."""
    n, L = spec.n, spec.levels
    px = [(spec.w >> l) * (spec.h >> l) for l in range(L)]
    tile = min(L, 6)
    pyr = n * (3 * px[0] + sum(px[:tile]))
    bit = n * (sum(px) + sum(px) / 4 + sum(px[tile:]))
    srch = spec.pairs * sum(px) / 2
    return {"pyramid": pyr, "bitmaps": bit, "search": srch}


def kernels_per_step(spec) -> int:
    return 4  # k_clear, k_pyramid, k_bitmaps, k_search


KERNEL_SOURCES = {  # the files each recorded kernel is built from
    "k_pyramid": ("mtb_pyramid.cu", "mtb_pyramid_dev.cuh", "mtb_device.cuh", "mtb_internal.cuh"),
    "k_bitmaps": ("mtb_bitmaps.cu", "mtb_bitmaps_dev.cuh", "mtb_device.cuh", "mtb_internal.cuh"),
    "k_search_staged": ("mtb_search.cu", "mtb_search_staged.cuh", "mtb_search_dev.cuh", "mtb_device.cuh",
                        "mtb_internal.cuh"),
    "k_search_items": ("mtb_search.cu", "mtb_search_dev.cuh", "mtb_device.cuh", "mtb_internal.cuh"),
    "k_apply_shifts": ("mtb_apply.cu", "mtb_internal.cuh"),
}
# the search stage runs one of two kernels (mtb_search_kernel tells which)
STAGE_KERNEL = {"pyramid": "k_pyramid", "bitmaps": "k_bitmaps", "search": "k_search_staged"}


def kernel_sources_digest(kernel: str) -> str:
    """SHA-256 over the CUDA sources a kernel is built from (and the C ABI
    header); any change voids a stored ncu figure."""
    csrc = os.path.join(ROOT, "paper_2007_06483_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(csrc, f), "rb").read())
    h.update(open(os.path.join(ROOT, "include", "mtb.h"), "rb").read())
    return h.hexdigest()


def traffic_for(kernel: str, workload: str):
    rec = NCU_TRAFFIC.get((kernel, workload))
    if not rec:
        return None
    return rec["bytes"] if rec["sources_sha256"] == kernel_sources_digest(kernel) else None


def hbm_peak():
    try:
        peaks = json.load(open(PEAKS_FILE))
        return float(peaks["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="mtb_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu=timestamp,{self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- CPU baseline
def host_cpu() -> dict:
    """The host the oracle baseline ran on: online cores, cores this process may
    use, architecture and CPU model (x86 `model name`; on Arm, where
    /proc/cpuinfo has none, lscpu's model name or the implementer/part codes)."""
    import platform

    info = {"nproc": os.cpu_count(), "usable_cores": len(os.sched_getaffinity(0)), "arch": platform.machine(),
            "model": None}
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                fields.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    info["model"] = fields.get("model name") or None
    if info["model"] is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.strip().startswith("Model name:"):
                    info["model"] = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    if info["model"] is None and "CPU implementer" in fields:
        info["model"] = f"implementer {fields['CPU implementer']} part {fields.get('CPU part', '?')}"
    return info


def oracle_rate(images_np, spec, budget_s: float = 12.0, max_s: float = 30.0) -> dict:
    """Single-threaded oracle on the same stack, repeated to about budget_s."""
    import oracle

    t0 = time.perf_counter()
    res = oracle.align_stack(images_np, spec.levels, spec.noise_tol, spec.ref)
    first = time.perf_counter() - t0
    reps = 1
    total = first
    while total + first <= min(budget_s, max_s):
        oracle.align_stack(images_np, spec.levels, spec.noise_tol, spec.ref)
        reps += 1
        total = time.perf_counter() - t0
    rate = spec.aligned_pixels * reps / total / 1e6
    return {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{reps} x full {spec.name} stack ({spec.pairs} pairs), single-threaded C oracle, {total:.1f} s",
            "host": host_cpu(), "result": res}


def oracle_rate_threaded(images_np, spec, threads: int, budget_s: float = 8.0) -> dict:
    """The same oracle on `threads` host threads at once, each aligning the whole
    stack again and again for about budget_s (the C oracle is reentrant and its
    calls release the GIL).  A reported baseline only, labelled with the thread
    count; the time runs until the last thread's last stack is done."""
    import threading

    import oracle

    oracle.align_stack(images_np, spec.levels, spec.noise_tol, spec.ref)  # library loaded
    done = [0] * threads
    t0 = time.perf_counter()
    stop = t0 + budget_s

    def work(i):
        while True:
            oracle.align_stack(images_np, spec.levels, spec.noise_tol, spec.ref)
            done[i] += 1
            if time.perf_counter() >= stop:
                return

    pool = [threading.Thread(target=work, args=(i,)) for i in range(threads)]
    for t in pool:
        t.start()
    for t in pool:
        t.join()
    total = time.perf_counter() - t0
    stacks = sum(done)
    return {"value": round(spec.aligned_pixels * stacks / total / 1e6, 3), "unit": UNIT, "cores": threads,
            "kind": "oracle", "sample": f"{stacks} x full {spec.name} stack on {threads} threads (each thread "
                                        f"aligns whole stacks), single-threaded C oracle per thread, {total:.1f} s",
            "host": host_cpu()}


def oracle_many(jobs, threads: int) -> list:
    """The single-threaded oracle over many stacks at once, one stack per task
    on `threads` host threads (the C oracle is reentrant and its calls release
    the GIL).  jobs: callables returning (images uint8 [n, h, w, 3] numpy,
    levels, noise_tol, ref); a job's host copy is made inside its task, so at
    most `threads` stacks are held in host memory at a time.  Returns each
    stack's oracle result in job order."""
    import concurrent.futures as cf

    import oracle

    oracle.default()  # loaded once, before the threads

    def one(job):
        imgs, levels, tol, ref = job()
        return oracle.align_stack(imgs, levels, tol, ref)

    with cf.ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
        return list(ex.map(one, jobs))


def usable_cores() -> int:
    return len(os.sched_getaffinity(0))


def batch_record(count: int, dev, stream, warmup: int, steps: int, oracle_check: bool = True,
                 sampler=None) -> dict:
    """Uneven stacks (synth.batch_specs) in one persistent graph-captured launch
    after the autotuner, against the plain per-stack path on the same stacks;
    every stack's shifts and per-level errors compared with the plain path and,
    when oracle_check, with the oracle (on every usable host core, outside the
    timed regions)."""
    import numpy as np
    import torch

    import paper_2007_06483_gb300 as mtb
    from paper_2007_06483_gb300 import synth

    specs = synth.batch_specs(count)
    stacks = [{"images": synth.make_stack(sp, dev), "levels": sp.levels, "noise_tol": sp.noise_tol,
               "ref_idx": sp.ref} for sp in specs]
    pixels = sum(sp.aligned_pixels for sp in specs)
    abytes = sum(sum(algorithmic_bytes(sp).values()) for sp in specs)
    t_tune = time.perf_counter()
    batch = mtb.Batch(stacks, level_outputs=True)
    batch.tune(reps=2, stream=stream)
    t_tune = time.perf_counter() - t_tune
    cfg = batch.config()
    for _ in range(max(3, warmup)):
        batch.run(stream)
    torch.cuda.synchronize(dev)
    K = max(1, steps)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    if sampler is not None:
        sampler.start()
    for k in range(K):
        evs[k][0].record(stream)
        batch.run(stream)
        evs[k][1].record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop() if sampler is not None else None
    status = batch.status()
    step_ms = [e[0].elapsed_time(e[1]) for e in evs]
    ms = evs[0][0].elapsed_time(evs[-1][1]) / K
    expected_ok = sum(np.array_equal(batch.shifts[k].cpu().numpy(), synth.expected_shifts(sp))
                      for k, sp in enumerate(specs))

    # the same stacks through the plain path, one stack after the other
    wss = [mtb.new_workspace(sp.n, sp.w, sp.h, sp.levels, device=dev) for sp in specs]
    outs = [torch.empty((sp.n, 2), dtype=torch.int32, device=dev) for sp in specs]

    def plain():
        for k, st in enumerate(stacks):
            mtb.align_stack(st["images"], st["levels"], st["noise_tol"], st["ref_idx"], workspace=wss[k],
                            out=outs[k], stream=stream)

    same = 0
    for k, st in enumerate(stacks):  # per-level outputs too, outside the timed runs
        r = mtb.align_stack(st["images"], st["levels"], st["noise_tol"], st["ref_idx"], level_outputs=True,
                            workspace=wss[k], stream=stream)
        same += int(torch.equal(r[0], batch.shifts[k]) and torch.equal(r[1], batch.level_errs[k]) and
                    torch.equal(r[2], batch.level_shifts[k]))
    torch.cuda.synchronize(dev)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Kp = max(1, min(K, 5))
    p0.record(stream)
    for _ in range(Kp):
        plain()
    p1.record(stream)
    torch.cuda.synchronize(dev)
    plain_ms = p0.elapsed_time(p1) / Kp
    rec = {"stacks": count, "exposures": sum(sp.n for sp in specs), "pairs": sum(sp.pairs for sp in specs),
           "aligned_mpix": round(pixels / 1e6, 1), "value": round(pixels / (ms / 1e3) / 1e6, 2), "unit": UNIT,
           "ms_per_run": round(ms, 4), "runs": K,
           "latency_ms": {"p50": round(_pct(step_ms, 0.50), 4), "p99": round(_pct(step_ms, 0.99), 4)},
           "plain_value": round(pixels / (plain_ms / 1e3) / 1e6, 2), "plain_ms_per_run": round(plain_ms, 4),
           "batch_vs_plain": round(plain_ms / ms, 3), "tile_shapes": cfg, "tune_s": round(t_tune, 2),
           "status_ok": status == mtb.MTB_OK, "equal_plain_path": f"{same}/{count}",
           "planted_shifts_recovered": f"{expected_ok}/{count} stacks",
           "alg_GBps": round(abytes / (ms / 1e3) / 1e9, 1), "algorithmic_bytes_per_run": abytes}
    if oracle_check:
        t = time.perf_counter()
        jobs = [(lambda k=k: (stacks[k]["images"].cpu().numpy(), specs[k].levels, specs[k].noise_tol,
                              specs[k].ref)) for k in range(count)]
        res = oracle_many(jobs, usable_cores())
        eq = sum(np.array_equal(batch.shifts[k].cpu().numpy(), r["shifts"]) and
                 np.array_equal(batch.level_errs[k].cpu().numpy().view(np.uint32), r["level_errs"]) and
                 np.array_equal(batch.level_shifts[k].cpu().numpy(), r["level_shifts"])
                 for k, r in enumerate(res))
        rec["oracle_equal"] = f"{eq}/{count}"
        rec["oracle_check"] = (f"shifts, per-level errors and per-level shifts of every stack vs the single-"
                               f"threaded C oracle on {usable_cores()} host threads, {time.perf_counter() - t:.1f} s")
    if clocks is not None:
        rec["clocks"] = clocks
    batch.close()
    del stacks, wss, outs
    torch.cuda.empty_cache()
    return rec


# ----------------------------------------------------------------------------- GPU arm
def run_gb300(args):
    import numpy as np
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else torch.cuda.current_device())
    torch.cuda.set_device(dev)

    from paper_2007_06483_gb300 import build as cuda_build

    cuda_build.build()
    import paper_2007_06483_gb300 as mtb
    from paper_2007_06483_gb300 import synth

    base = workload(args.workload)
    units = shard_units(world, rank, world)  # one stack per rank per step
    spec = dataclasses.replace(base, seed=base.seed + 1000 * units[0]) if units[0] else base
    n, w, h, L = spec.n, spec.w, spec.h, spec.levels
    images = synth.make_stack(spec, dev)
    B = max(1, args.buffers)
    imgs = [images] + [images.clone() for _ in range(B - 1)]
    wss = [mtb.new_workspace(n, w, h, L, device=dev) for _ in range(B)]
    shifts = [torch.empty((n, 2), dtype=torch.int32, device=dev) for _ in range(B)]
    stream = torch.cuda.current_stream(dev)

    def step(b, ev=None):
        if ev is not None:
            ev[0].record(stream)
        mtb.align_stack(imgs[b], L, spec.noise_tol, spec.ref, workspace=wss[b], out=shifts[b], stream=stream)
        if ev is not None:
            ev[1].record(stream)

    def staged(b, ev):
        ev[0].record(stream)
        mtb.build_pyramids(imgs[b], L, wss[b], stream)
        ev[1].record(stream)
        mtb.build_bitmaps(n, w, h, L, spec.noise_tol, wss[b], stream)
        ev[2].record(stream)
        mtb.search_shifts(n, w, h, L, spec.ref, wss[b], shifts[b], None, None, stream)
        ev[3].record(stream)

    if args.profile_steps > 0:  # a short run for profilers: plain steps only, nothing timed or printed
        for k in range(args.profile_steps):
            step(k % B)
        torch.cuda.synchronize(dev)
        return

    for k in range(max(3, args.warmup)):
        step(k % B)
    torch.cuda.synchronize(dev)

    # throughput: K steps back to back between two events (an event between
    # two steps would end the overlap of one step's search with the next
    # step's launches); that region again and again, each time between a
    # barrier and a synchronize, until the regions add up to min_timed_s
    K = args.steps
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    sampler.start()
    total_ms, t_wall, regions = 0.0, 0.0, 0
    while True:
        barrier(world)
        torch.cuda.synchronize(dev)
        tw = time.perf_counter()
        t0.record(stream)
        for k in range(K):
            step(k % B)
        t1.record(stream)
        torch.cuda.synchronize(dev)
        t_wall += time.perf_counter() - tw
        barrier(world)
        total_ms += max_over_ranks(t0.elapsed_time(t1), world, dev)
        regions += 1
        # every rank takes the same decision: the max over ranks of the wall time
        if max_over_ranks(t_wall, world, dev) >= args.min_timed_s:
            break
    clocks = sampler.stop()
    ms_per_step = total_ms / (K * regions)

    # latency: max(LAT_STEPS, K) steps, each between its own two events, after
    # LAT_WARMUP more untimed ones
    for k in range(LAT_WARMUP):
        step(k % B)
    n_lat = max(LAT_STEPS, K)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(n_lat)]
    for k in range(n_lat):
        step(k % B, evs[k])
    torch.cuda.synchronize(dev)
    step_ms = [e[0].elapsed_time(e[1]) for e in evs]

    # the same work through the three stage calls, for the split by stage
    sev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(max(3, K))]
    for k in range(3):
        staged(k % B, sev[k])
    for k, ev in enumerate(sev):
        staged(k % B, ev)
    torch.cuda.synchronize(dev)
    stage_ms = {
        "pyramid": statistics.mean(e[0].elapsed_time(e[1]) for e in sev),
        "bitmaps": statistics.mean(e[1].elapsed_time(e[2]) for e in sev),
        "search": statistics.mean(e[2].elapsed_time(e[3]) for e in sev),
    }
    value = world * spec.aligned_pixels / (ms_per_step / 1e3) / 1e6

    # correctness of what was timed: every buffer's shifts vs the planted ones
    want = synth.expected_shifts(spec)
    got = shifts[0].cpu().numpy()
    same_all = all(torch.equal(s, shifts[0]) for s in shifts)
    planted_ok = (f"{int((got == want).all(axis=1).sum())}/{n} exposures" +
                  ("" if same_all else ", buffers disagree"))

    abytes = algorithmic_bytes(spec)
    peak, peak_kind = hbm_peak()
    step_bytes = sum(abytes.values())
    # the dominant kernel is the stage with the largest share of the staged
    # split; its duration is that stage between CUDA events on the launching
    # stream (the pyramid stage's k_clear is a few-KB clear overlapped by PDL,
    # the search stage's k_clear_search likewise)
    staged_total = sum(stage_ms.values())
    top = max(stage_ms, key=stage_ms.get)
    achieved = abytes[top] / (stage_ms[top] / 1e3) / 1e9
    call = {"pyramid": "mtb_build_pyramids", "bitmaps": "mtb_build_bitmaps", "search": "mtb_search_shifts"}
    kern = dict(STAGE_KERNEL)
    kern["search"] = "k_search_" + mtb.search_kernel(n, w, h, L, spec.ref, chained=False)
    roofline = {"bound": "hbm", "kernel": kern[top], "achieved": round(achieved, 1), "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": traffic_for(kern[top], spec.name), "algorithmic_bytes_per_launch": abytes[top],
                "ms_per_launch": round(stage_ms[top], 5),
                "share_of_staged_step": round(stage_ms[top] / staged_total, 3),
                "duration_source": f"CUDA events around {call[top]}, {len(sev)} staged steps after the "
                                   f"timed region, same buffers and stream"}
    stages = {k: {"kernel": kern[k], "ms": round(v, 5), "share": round(v / staged_total, 3),
                  "alg_GBps": round(abytes[k] / (v / 1e3) / 1e9, 1),
                  "frac_of_peak": round(abytes[k] / (v / 1e3) / 1e9 / peak, 4),
                  "traffic": traffic_for(kern[k], spec.name)} for k, v in stage_ms.items()}

    # ---- end to end through the host-buffer entry point ----
    e2e = None
    if not args.no_e2e:
        host = images.cpu().pin_memory()
        dws = torch.empty(mtb.host_workspace_bytes(n, w, h, L), dtype=torch.uint8, device=dev)
        host_out = torch.empty((n, 2), dtype=torch.int32, pin_memory=True)
        for _ in range(2):
            mtb.align_stack_host(host, L, spec.noise_tol, spec.ref, device_workspace=dws, out=host_out,
                                 stream=stream)
        Ke = max(3, min(K, 20))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(world)
        e0.record(stream)
        for _ in range(Ke):
            out = mtb.align_stack_host(host, L, spec.noise_tol, spec.ref, device_workspace=dws, out=host_out,
                                       stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        e_ms = max_over_ranks(e0.elapsed_time(e1) / Ke, world, dev)
        e2e_same = np.array_equal(out.numpy(), got)
        e2e = {"value": round(world * spec.aligned_pixels / (e_ms / 1e3) / 1e6, 2), "unit": UNIT,
               "ms_per_step": round(e_ms, 4), "h2d_bytes_per_step": int(host.numel()),
               "d2h_bytes_per_step": int(out.numel() * out.element_size()), "steps": Ke,
               "shifts_equal_device_path": bool(e2e_same)}

    cpu = cpu_threaded = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res = oracle_rate(images.cpu().numpy(), spec)
        gpu_match = all(np.array_equal(s.cpu().numpy(), res["result"]["shifts"]) for s in shifts)
        g_s, g_e, g_l = mtb.align_stack(images, L, spec.noise_tol, spec.ref, level_outputs=True, workspace=wss[0],
                                        stream=stream)
        levels_match = (np.array_equal(g_e.cpu().numpy().view(np.uint32), res["result"]["level_errs"]) and
                        np.array_equal(g_l.cpu().numpy(), res["result"]["level_shifts"]))
        cpu = {k: v for k, v in res.items() if k != "result"}
        cpu["value"] = round(cpu["value"], 3)
        cpu["gpu_shifts_equal_oracle"] = bool(gpu_match)
        cpu["gpu_level_errors_and_shifts_equal_oracle"] = bool(levels_match)
        if args.cpu_threads != 1:
            nthr = args.cpu_threads if args.cpu_threads > 0 else len(os.sched_getaffinity(0))
            cpu_threaded = oracle_rate_threaded(images.cpu().numpy(), spec, nthr)

    batch = None
    if rank == 0 and world == 1 and args.batch_count > 0:
        batch = batch_record(args.batch_count, dev, stream, args.warmup, 5,
                             oracle_check=not args.no_cpu_baseline)

    serve = None
    if rank == 0 and world == 1 and args.serve_pool > 0:
        # a short served run (10, 100 and 1000 jobs/s offered, 64 jobs each)
        # of 6000x4000x7 jobs, every result checked against the oracle
        sargs = argparse.Namespace(**vars(args))
        sargs.pool, sargs.rates = args.serve_pool, "10,100,1000"
        serve = serve_summary(serve_line(sargs, max_jobs=64, probe=False))

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": plain_config(spec, world, B),
            "l2_bytes_rotated": B * (spec.input_bytes + wss[0].numel()),
            "latency_ms": {"p50": round(_pct(step_ms, 0.50), 5), "p99": round(_pct(step_ms, 0.99), 5),
                           "runs": len(step_ms), "warmup": LAT_WARMUP},
            "hbm_gbs": round(step_bytes / (ms_per_step / 1e3) / 1e9, 1),
            "stages": stages,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "cpu_baseline_threaded": cpu_threaded,
            "e2e": e2e,
            "batch": batch,
            "serve": serve,
            "gpu_launches": K * regions * kernels_per_step(spec),
            "clocks": clocks,
            "planted_shifts_recovered": planted_ok,
            "timed_regions": regions,
            "wall_s_timed_region": round(t_wall, 4),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle as it stands, on the host cores, on the same workload, metric
    and unit as the GPU arm: a step aligns the whole stack (every exposure's
    pyramid built, every pair searched), on the same input bytes the GPU arm
    aligns (the stack is generated on the GPU when there is one, as the GPU arm
    does, and copied to the host).  If K + W whole stacks would take more than
    about 150 s, every exposure is cropped to its first rows, and the line says
    so."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    import torch

    import oracle
    from paper_2007_06483_gb300 import synth

    spec = workload(args.workload)
    gen_dev = "cuda" if torch.cuda.is_available() else "cpu"
    images = synth.make_stack(spec, gen_dev).cpu().numpy()
    t = time.perf_counter()
    oracle.align_stack(images, spec.levels, spec.noise_tol, spec.ref)
    one = time.perf_counter() - t
    budget = 150.0
    rows = spec.h
    if one * (args.steps + args.warmup) > budget:
        rows = max(1 << (spec.levels - 1), int(spec.h * budget / (one * (args.steps + args.warmup))))
        images = np.ascontiguousarray(images[:, :rows])
    for _ in range(args.warmup):
        oracle.align_stack(images, spec.levels, spec.noise_tol, spec.ref)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.align_stack(images, spec.levels, spec.noise_tol, spec.ref)
    dt = (time.perf_counter() - t) / args.steps
    px = spec.pairs * spec.w * rows
    value = px / dt / 1e6
    crop = "" if rows == spec.h else f", cropped to the first {rows} of {spec.h} rows"
    sample = (f"the whole {spec.name} stack ({spec.pairs} pairs) per step{crop}, single-threaded C oracle, "
              f"inputs generated on {gen_dev} as the GPU arm's")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": plain_config(spec, args.gpus, max(1, args.buffers)),
        "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "host": host_cpu()},
        "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- batched form
def run_batch(args):
    """Uneven stacks (synth.batch_specs) in one persistent graph-captured launch,
    after the autotuner picked its tile shapes; the same stacks through the
    plain per-stack path for comparison, and every stack checked against the
    plain path and the oracle.  A step aligns every stack once."""
    import torch

    from paper_2007_06483_gb300 import build as cuda_build

    cuda_build.build()

    count = int(args.workload[len("batch"):] or 256)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    rec = batch_record(count, dev, stream, args.warmup, args.steps, oracle_check=not args.no_cpu_baseline,
                       sampler=ClockSampler(dev.index or 0))
    peak, peak_kind = hbm_peak()
    achieved = rec["alg_GBps"]
    line = {
        "metric": METRIC + " (batched)", "value": rec["value"], "unit": UNIT, "n_gpus": 1,
        "steps": rec["runs"], "warmup": args.warmup, "ms_per_step": rec["ms_per_run"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"batch{count}", "stacks": count, "exposures": rec["exposures"],
                   "pairs": rec["pairs"], "aligned_mpix": rec["aligned_mpix"], "tile_shapes": rec["tile_shapes"],
                   "l2": "inputs of the batch far exceed L2"},
        "plain_path": {"value": rec["plain_value"], "ms_per_step": rec["plain_ms_per_run"],
                       "equal_plain_path": rec["equal_plain_path"]},
        "batch_vs_plain": rec["batch_vs_plain"],
        "oracle_equal": rec.get("oracle_equal"), "oracle_check": rec.get("oracle_check"),
        "latency_ms": rec["latency_ms"],
        "hbm_gbs": achieved,
        "roofline": {"bound": "hbm", "kernel": "k_engine<batch> (after k_engine_clear)", "achieved": achieved,
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": None, "algorithmic_bytes_per_launch": rec["algorithmic_bytes_per_run"]},
        "gpu_launches": 2 * rec["runs"], "clocks": rec.get("clocks"),
        "planted_shifts_recovered": rec["planted_shifts_recovered"],
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- serving
def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, max(0, int(math.ceil(q * len(xs))) - 1))]


def h2d_link_gbs(host, dev, stream, reps: int = 5) -> float:
    """Host-to-device copy bandwidth of this machine's link, from pinned memory."""
    import torch

    d = torch.empty(host.shape, dtype=host.dtype, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(reps):
        e0.record(stream)
        d.copy_(host, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        best = min(best, e0.elapsed_time(e1))
    del d
    return host.numel() / (best / 1e3) / 1e9


def h2d_copy_probe(pool, dev, stream, count: int = 40, gap_s: float = 0.02) -> dict:
    """Single 504 MB pinned host-to-device transfers, one at a time and `gap_s`
    apart (a low offered load), each timed with CUDA events, with no alignment
    and no server around them: by a copy engine (cudaMemcpyAsync) and by SM
    loads (a PyTorch elementwise kernel reading the pinned buffer through
    unified addressing, as the server's copy kernel does).  A copy engine idle
    for milliseconds is slow to start its next copy; SM loads are not."""
    import torch

    class _Cai:  # the pinned buffer as a device array at the same address
        def __init__(self, t):
            self.__cuda_array_interface__ = {"shape": (t.numel() // 8,), "typestr": "<i8",
                                             "data": (t.data_ptr(), False), "version": 3}

    d = torch.empty(pool[0].shape, dtype=pool[0].dtype, device=dev)
    d64 = d.view(-1).view(torch.int64)
    views = [torch.as_tensor(_Cai(p), device=dev) if p.is_pinned() and p.numel() % 8 == 0 else None for p in pool]
    out = {}
    for mode in ("copy_engine", "sm_loads"):
        ms = []
        for k in range(count):
            src = pool[k % len(pool)]
            v = views[k % len(pool)]
            if mode == "sm_loads" and v is None:
                continue
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if mode == "copy_engine":
                d.copy_(src, non_blocking=True)
            else:
                torch.bitwise_or(v, 0, out=d64)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
            time.sleep(gap_s)
        if ms:
            out[mode] = {"copies": len(ms), "gap_ms": gap_s * 1e3, "p50_ms": round(_pct(ms, 0.50), 3),
                         "p99_ms": round(_pct(ms, 0.99), 3), "max_ms": round(max(ms), 3)}
    del d
    return out


def run_serve(args):
    print(json.dumps(serve_line(args)), flush=True)


def serve_line(args, max_jobs: int = 500, probe: bool = True) -> dict:
    """Poisson arrivals of 6000x4000x7 jobs (synth.serve_specs, pinned host
    memory) into the serving loop under a device-memory budget, swept over the
    offered rates (at most max_jobs jobs a rate).  Latency runs from a job's
    scheduled arrival to its shifts being in host memory (copy in over
    NVLink-C2C, alignment, copy out).  Every served result is compared with the
    same job aligned alone on the plain path and with the oracle's answer."""
    import threading

    import numpy as np
    import torch

    from paper_2007_06483_gb300 import build as cuda_build

    cuda_build.build()
    import paper_2007_06483_gb300 as mtb
    from paper_2007_06483_gb300 import synth

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    specs = synth.serve_specs(args.pool)
    pool, alone, planted, resident = [], [], 0, []
    for sp in specs:
        d = synth.make_stack(sp, dev)
        h = torch.empty(d.shape, dtype=torch.uint8, pin_memory=True)
        h.copy_(d)
        out = mtb.align_stack(d, sp.levels, sp.noise_tol, sp.ref, stream=stream)
        pool.append(h)
        resident.append(d)
        alone.append(out.cpu())
        planted += int(np.array_equal(alone[-1].numpy(), synth.expected_shifts(sp)))
    # every job's answer from the oracle, on every usable host core (outside the timed sweep)
    t_orc = time.perf_counter()
    orc = None
    if not args.no_cpu_baseline:
        res = oracle_many([(lambda h=h, sp=sp: (h.numpy(), sp.levels, sp.noise_tol, sp.ref))
                           for h, sp in zip(pool, specs)], usable_cores())
        orc = [torch.from_numpy(r["shifts"].astype(np.int32)) for r in res]
    t_orc = time.perf_counter() - t_orc
    # the plain path on the same jobs, inputs already in HBM, for comparison
    ws = mtb.new_workspace(specs[0].n, specs[0].w, specs[0].h, specs[0].levels, device=dev)
    outp = torch.empty((specs[0].n, 2), dtype=torch.int32, device=dev)
    for d in resident[:3]:
        mtb.align_stack(d, specs[0].levels, specs[0].noise_tol, specs[0].ref, workspace=ws, out=outp, stream=stream)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for d in resident:
        mtb.align_stack(d, specs[0].levels, specs[0].noise_tol, specs[0].ref, workspace=ws, out=outp, stream=stream)
    p1.record(stream)
    torch.cuda.synchronize(dev)
    plain_ms = p0.elapsed_time(p1)
    del resident, ws, outp
    torch.cuda.empty_cache()
    link_gbs = h2d_link_gbs(pool[0], dev, stream)
    copy_probe = h2d_copy_probe(pool, dev, stream) if probe else None
    sp0 = specs[0]
    px = sp0.aligned_pixels
    job_bytes = mtb.job_bytes(sp0.n, sp0.w, sp0.h, sp0.levels, sp0.noise_tol, sp0.ref)
    budget = int(args.budget_gb * 1e9)
    rates = [float(r) for r in args.rates.split(",") if r]
    rng = np.random.default_rng(17)
    results, all_same = [], True
    sampler = ClockSampler(dev.index or 0)
    with mtb.Server(budget, slots=args.slots, copy_streams=args.copy_streams) as srv:
        # warm-up: a few jobs through the server
        for k in range(max(3, args.warmup)):
            srv.wait(srv.submit(pool[k % len(pool)], sp0.levels, sp0.noise_tol, sp0.ref))
        sampler.start()
        for rate in rates:
            count = int(min(max_jobs, max(64, min(500, rate * 3))))
            gaps = rng.exponential(1.0 / rate, count)
            sched = np.cumsum(gaps) - gaps[0]
            picks = [k % len(pool) for k in range(count)]
            ids, slip = [None] * count, [0.0] * count
            t0 = time.perf_counter() + 0.05

            def submitter():
                for i in range(count):
                    target = t0 + sched[i]
                    while True:
                        now = time.perf_counter()
                        if now >= target:
                            break
                        if target - now > 0.002:
                            time.sleep(target - now - 0.001)
                    slip[i] = time.perf_counter() - target
                    try:
                        ids[i] = srv.submit(pool[picks[i]], sp0.levels, sp0.noise_tol, sp0.ref)
                    except Exception as exc:  # surfaces in the main thread
                        ids[i] = exc
                        return

            th = threading.Thread(target=submitter)
            th.start()
            lat, queue, done_at = [], [], []
            phases = {"enqueue": [], "device": [], "callback": []}
            same = orc_same = 0
            for i in range(count):
                while ids[i] is None:
                    time.sleep(0.0002)
                if isinstance(ids[i], Exception):
                    raise ids[i]
                shifts, ph = srv.wait_phases(ids[i])
                l_ms, q_ms = ph["total"], ph["queue"]
                for k in phases:
                    phases[k].append(ph[k])
                l_ms += slip[i] * 1e3  # from the scheduled arrival
                lat.append(l_ms)
                queue.append(q_ms + slip[i] * 1e3)
                done_at.append(sched[i] + l_ms / 1e3)
                same += int(torch.equal(shifts, alone[picks[i]]))
                orc_same += int(orc is not None and torch.equal(shifts, orc[picks[i]]))
            th.join()
            st = srv.stats()
            span = max(done_at)
            all_same = all_same and same == count
            results.append({
                "offered_jobs_s": rate, "jobs": count, "served_jobs_s": round(count / span, 2),
                "mpix_s": round(count * px / span / 1e6, 1),
                "h2d_gbs": round(count * sp0.input_bytes / span / 1e9, 1),
                "p50_ms": round(_pct(lat, 0.50), 3), "p99_ms": round(_pct(lat, 0.99), 3),
                "queue_p50_ms": round(_pct(queue, 0.50), 3), "queue_p99_ms": round(_pct(queue, 0.99), 3),
                "submit_slip_p99_ms": round(_pct(slip, 0.99) * 1e3, 3),
                # where the latency goes (host clock): enqueueing the job's work,
                # the copy in + alignment + copy out + callback dispatch, the callback
                "phases_p50_p99_ms": {k: [round(_pct(v, 0.50), 3), round(_pct(v, 0.99), 3)]
                                      for k, v in phases.items()},
                "same_as_alone": f"{same}/{count}",
                "oracle_equal": f"{orc_same}/{count}" if orc is not None else None,
            })
        clocks = sampler.stop()
        st = srv.stats()
    best = max(results, key=lambda r: r["mpix_s"])
    line = {
        "metric": METRIC + " (served)", "value": best["mpix_s"], "unit": UNIT, "n_gpus": 1,
        "steps": sum(r["jobs"] for r in results), "warmup": max(3, args.warmup),
        "ms_per_step": round(1e3 / best["served_jobs_s"], 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": "serve6000x4000x7", "pool_jobs": len(pool), "w": sp0.w, "h": sp0.h,
                   "n_exposures": sp0.n, "levels": sp0.levels, "budget_gb": args.budget_gb,
                   "job_gb": round(job_bytes / 1e9, 3), "slots": args.slots, "copy_streams": args.copy_streams,
                   "arrivals": "Poisson, seeded", "l2": "every job's 504 MB input comes over NVLink-C2C"},
        "serving": results,
        "plain_path_device_resident": {"mpix_s": round(px * len(specs) / (plain_ms / 1e3) / 1e6, 1),
                                        "ms_per_job": round(plain_ms / len(specs), 4)},
        "e2e": {"value": best["mpix_s"], "unit": UNIT, "h2d_bytes_per_step": int(sp0.input_bytes),
                "d2h_bytes_per_step": int(sp0.n * 8)},
        "roofline": {"bound": "h2d_link", "kernel": "k_copy_in (SM loads of pinned host memory over NVLink-C2C)",
                     "achieved": best["h2d_gbs"], "peak": round(link_gbs, 1),
                     "peak_kind": "measured in this run: best of 5 pinned 504 MB host->device copies",
                     "unit": "GB/s", "frac": round(best["h2d_gbs"] / link_gbs, 4), "traffic": None},
        "server_stats": st,
        # the device phase's tail comes from the copy in: the same copies
        # alone, spaced like a low offered load
        "h2d_copy_alone": copy_probe,
        "results_same_alone_and_in_mix": bool(all_same),
        "alone_equal_oracle": (f"{sum(torch.equal(a, o) for a, o in zip(alone, orc))}/{len(alone)}"
                               if orc is not None else None),
        "oracle_check": (f"every served job's shifts vs the single-threaded C oracle's answer for its pool job "
                         f"({len(pool)} jobs on {usable_cores()} host threads, {t_orc:.1f} s, before the sweep)"
                         if orc is not None else None),
        "planted_shifts_recovered": f"{planted}/{len(specs)} jobs",
        "gpu_launches": kernels_per_step(sp0) * sum(r["jobs"] for r in results), "clocks": clocks,
    }
    del pool, srv
    torch.cuda.empty_cache()
    return line


def serve_summary(line: dict) -> dict:
    """The served form in brief, for the default line: per offered rate the
    served rate, latency and the equality counts, and the best served MPix/s
    against the plain path on the same jobs."""
    best = line["value"]
    plain = line["plain_path_device_resident"]["mpix_s"]
    return {
        "workload": line["config"]["workload"], "pool_jobs": line["config"]["pool_jobs"],
        "slots": line["config"]["slots"], "budget_gb": line["config"]["budget_gb"],
        "value": best, "unit": line["unit"], "plain_device_resident_mpix_s": plain,
        "served_vs_plain": round(best / plain, 4) if plain else None,
        "h2d_link_frac": line["roofline"]["frac"],
        "rates": [{k: r[k] for k in ("offered_jobs_s", "jobs", "served_jobs_s", "mpix_s", "p50_ms", "p99_ms",
                                      "same_as_alone", "oracle_equal")} for r in line["serving"]],
        "alone_equal_oracle": line["alone_equal_oracle"], "oracle_check": line["oracle_check"],
        "server_stats": line["server_stats"],
    }


# ----------------------------------------------------------------------------- after the alignment
def _time_calls(fn, K: int, W: int, stream, dev) -> float:
    """Mean ms of fn() over K calls after W, CUDA events on the launching stream."""
    import torch

    for _ in range(max(3, W)):
        fn()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        fn()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) / K


def run_apply(args):
    """mtb_apply_shifts on the 6000x4000x7 stack with its own shifts: every
    exposure moved (edge fill), 3 bytes read and 3 written per pixel."""
    import torch

    from paper_2007_06483_gb300 import build as cuda_build

    cuda_build.build()
    import paper_2007_06483_gb300 as mtb
    from paper_2007_06483_gb300 import synth

    spec = synth.STACK_24MP
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    imgs = synth.make_stack(spec, dev)
    shifts = mtb.align_stack(imgs, spec.levels, spec.noise_tol, spec.ref, stream=stream)
    outs = [torch.empty_like(imgs) for _ in range(2)]  # 2 x 504 MB: each step misses L2
    k = [0]

    def step():
        mtb.apply_shifts(imgs, shifts, mtb.MTB_FILL_EDGE, out=outs[k[0] % 2], stream=stream)
        k[0] += 1

    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    ms = _time_calls(step, args.steps, args.warmup, stream, dev)
    clocks = sampler.stop()
    px = spec.n * spec.w * spec.h
    moved = 2 * spec.input_bytes
    peak, peak_kind = hbm_peak()
    achieved = moved / (ms / 1e3) / 1e9
    line = {
        "metric": "moved MPix/s (all exposures, RGB)", "value": round(px / (ms / 1e3) / 1e6, 1), "unit": "MPix/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": "apply6000x4000x7", "fill": "edge", "l2": "504 MB in, 2 x 504 MB out (> L2)"},
        "roofline": {"bound": "hbm", "kernel": "k_apply_shifts", "achieved": round(achieved, 1), "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic_for("k_apply_shifts", "apply6000x4000x7"),
                     "algorithmic_bytes_per_launch": moved},
        "gpu_launches": args.steps, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_paper(args):
    """The paper's measurement shape (Sec. IV): 2560x1440 stacks of 2..7
    exposures, timed end to end from pinned host memory (copy in, align, shifts
    out), as the paper includes the CPU-to-GPU transfer, and with the inputs
    already on the device; the chain mode, the quadrant test and moving the
    exposures are timed beside.  The oracle on one host core gives the context
    the paper's CPU column gives."""
    import numpy as np
    import torch

    from paper_2007_06483_gb300 import build as cuda_build

    cuda_build.build()
    import paper_2007_06483_gb300 as mtb
    from paper_2007_06483_gb300 import synth

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    K, W = args.steps, args.warmup
    rows = []
    for spec in synth.paper_specs():
        n, w, h, L = spec.n, spec.w, spec.h, spec.levels
        imgs = synth.make_stack(spec, dev)
        host = imgs.cpu().pin_memory()
        ws = mtb.new_workspace(n, w, h, L, device=dev)
        dws = torch.empty(mtb.host_workspace_bytes(n, w, h, L), dtype=torch.uint8, device=dev)
        qws = torch.empty(mtb.lib().mtb_quadrant_workspace_bytes(n, w, h, L - 1), dtype=torch.uint8, device=dev)
        out = torch.empty((n, 2), dtype=torch.int32, device=dev)
        host_out = torch.empty((n, 2), dtype=torch.int32, pin_memory=True)
        moved = torch.empty_like(imgs)
        t = {}
        t["e2e_ms"] = _time_calls(lambda: mtb.align_stack_host(host, L, spec.noise_tol, spec.ref,
                                                               device_workspace=dws, out=host_out, stream=stream),
                                  K, W, stream, dev)
        t["device_ms"] = _time_calls(lambda: mtb.align_stack(imgs, L, spec.noise_tol, spec.ref, workspace=ws, out=out,
                                                             stream=stream), K, W, stream, dev)
        t["chain_ms"] = _time_calls(lambda: mtb.align_stack_chain(imgs, L, spec.noise_tol, spec.ref, workspace=ws,
                                                                  out=out, stream=stream), K, W, stream, dev)
        t["quadrants_ms"] = _time_calls(lambda: mtb.align_quadrants(imgs, L - 1, spec.noise_tol, spec.ref, 1,
                                                                    workspace=qws, stream=stream), K, W, stream, dev)
        t["apply_ms"] = _time_calls(lambda: mtb.apply_shifts(imgs, out, mtb.MTB_FILL_EDGE, out=moved, stream=stream),
                                    K, W, stream, dev)
        shifts = mtb.align_stack(imgs, L, spec.noise_tol, spec.ref, stream=stream).cpu().numpy()
        row = {"n": n, **{k: round(v, 4) for k, v in t.items()},
               "e2e_mpix_s": round(spec.aligned_pixels / (t["e2e_ms"] / 1e3) / 1e6, 1),
               "device_mpix_s": round(spec.aligned_pixels / (t["device_ms"] / 1e3) / 1e6, 1),
               "planted_recovered": bool(np.array_equal(shifts, synth.expected_shifts(spec)))}
        if not args.no_cpu_baseline:
            import oracle

            t0 = time.perf_counter()
            res = oracle.align_stack(host.numpy(), L, spec.noise_tol, spec.ref)
            cpu_ms = (time.perf_counter() - t0) * 1e3
            row["oracle_1core_ms"] = round(cpu_ms, 1)
            row["e2e_speedup_vs_oracle"] = round(cpu_ms / t["e2e_ms"], 1)
            row["gpu_equals_oracle"] = bool(np.array_equal(shifts, res["shifts"]))
        rows.append(row)
        del imgs, host, ws, dws, qws, moved
    last = rows[-1]
    line = {
        "metric": METRIC + " (end to end, paper shape)", "value": last["e2e_mpix_s"], "unit": UNIT, "n_gpus": 1,
        "steps": K, "warmup": W, "ms_per_step": last["e2e_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": "paper2560x1440x2..7", "levels": 6, "quadrant_levels": 5,
                   "e2e": "pinned host -> device copy, alignment, shifts -> host"},
        "per_n": rows,
        "e2e": {"value": last["e2e_mpix_s"], "unit": UNIT, "h2d_bytes_per_step": 7 * 2560 * 1440 * 3,
                "d2h_bytes_per_step": 7 * 8},
        "cpu_baseline": None if args.no_cpu_baseline else {
            "value": round(synth.paper_specs()[-1].aligned_pixels / (last["oracle_1core_ms"] / 1e3) / 1e6, 2),
            "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "one run per stack size, single-threaded C oracle",
            "host": host_cpu()},
        "gpu_launches": kernels_per_step(None) * K,
    }
    print(json.dumps(line), flush=True)


def run_profile(args):
    """The plain workload's kernels and nothing else, as the target of ncu
    captures: W one-call steps (k_clear, k_pyramid, k_bitmaps, k_search_items),
    then K one-call steps, then K stage-split steps (k_pyramid, k_bitmaps,
    k_clear_search + the search kernel the library picks for the stage)."""
    import torch

    from paper_2007_06483_gb300 import build as cuda_build

    cuda_build.build()
    import paper_2007_06483_gb300 as mtb
    from paper_2007_06483_gb300 import synth

    spec = workload(args.workload)
    n, w, h, L = spec.n, spec.w, spec.h, spec.levels
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    images = synth.make_stack(spec, dev)
    ws = mtb.new_workspace(n, w, h, L, device=dev)
    out = torch.empty((n, 2), dtype=torch.int32, device=dev)
    for _ in range(args.warmup + args.steps):
        mtb.align_stack(images, L, spec.noise_tol, spec.ref, workspace=ws, out=out, stream=stream)
    for _ in range(args.steps):
        mtb.build_pyramids(images, L, ws, stream)
        mtb.build_bitmaps(n, w, h, L, spec.noise_tol, ws, stream)
        mtb.search_shifts(n, w, h, L, spec.ref, ws, out, None, None, stream)
    torch.cuda.synchronize(dev)
    print(json.dumps({"profile": spec.name, "search_kernel": mtb.search_kernel(n, w, h, L, spec.ref),
                      "shifts": out.cpu().tolist()}), flush=True)


def main(argv=None):
    args = parse_args(argv)
    if args.profile:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload.startswith("batch"):
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "apply":
        run_apply(args)
    elif args.workload == "paper":
        run_paper(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
