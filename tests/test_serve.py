"""Serving: jobs admitted continuously under a device-memory budget.  Each job's
shifts must be the same alone (plain path), in the mix, and in the oracle, bit
for bit; the arena never holds more than the budget; refused jobs are refused
before anything is queued."""
import ctypes
import threading
import time

import numpy as np
import pytest
import torch

from paper_2007_06483_gb300 import synth

# (w, h, n, levels, ref): uneven shapes, so jobs of different sizes share the arena
MIX = [
    (640, 480, 2, 6, 0), (1000, 700, 3, 5, 1), (257, 33, 2, 6, 0), (1001, 333, 5, 4, 3), (800, 600, 6, 7, 3),
    (2, 2, 2, 2, 1), (1024, 1024, 2, 11, 0), (333, 222, 3, 5, 1), (1500, 1000, 4, 7, 2), (37, 23, 2, 3, 1),
]


def _jobs():
    out = []
    for j, (w, h, n, L, ref) in enumerate(MIX):
        spec = synth.small_spec(700 + j, w, h, n=n, levels=L, shift_range=min(6, (1 << L) - 1), ref=ref)
        out.append((synth.make_stack(spec).pin_memory() if torch.cuda.is_available() else synth.make_stack(spec),
                    L, ref))
    return out


# ---------------------------------------------------------------- host-only checks
@pytest.mark.parametrize("budget,slots,copies,pending", [
    (1 << 19, 4, 1, 0),   # budget below 1 MiB
    (1 << 30, 0, 1, 0),
    (1 << 30, 65, 1, 0),
    (1 << 30, 4, 0, 0),
    (1 << 30, 4, 9, 0),
    (1 << 30, 4, 1, -1),
])
def test_server_config_rejected_on_host(mtb_lib, budget, slots, copies, pending):
    cfg = mtb_lib.ServerConfig(budget, slots, copies, pending)
    h = ctypes.c_void_p()
    assert mtb_lib.lib().mtb_server_create(ctypes.byref(cfg), ctypes.byref(h)) == mtb_lib.MTB_ERR_INVALID_ARG
    assert not h.value
    assert mtb_lib.lib().mtb_server_create(None, ctypes.byref(h)) == mtb_lib.MTB_ERR_INVALID_ARG


def test_job_bytes_is_the_host_entry_footprint(mtb_lib):
    for (w, h, n, L, ref) in MIX:
        assert mtb_lib.job_bytes(n, w, h, L, 4, ref) == mtb_lib.host_workspace_bytes(n, w, h, L) > 0
    assert mtb_lib.job_bytes(2, 64, 64, 8) == 0       # coarsest level empty
    assert mtb_lib.job_bytes(2, 64, 64, 3, 4, 2) == 0  # ref out of range
    assert mtb_lib.job_bytes(2, 64, 64, 3, 300) == 0   # tolerance out of range
    lib = mtb_lib.lib()
    assert lib.mtb_job_bytes(None) == 0
    jid = ctypes.c_uint64()
    job = mtb_lib.Job(1 << 20, 2, 64, 64, 3, 4, 0, 1 << 20)
    assert lib.mtb_server_submit(None, ctypes.byref(job), ctypes.byref(jid)) == mtb_lib.MTB_ERR_INVALID_ARG
    assert lib.mtb_server_poll(None, 1) == mtb_lib.MTB_ERR_INVALID_ARG
    assert lib.mtb_server_wait(None, 1, None) == mtb_lib.MTB_ERR_INVALID_ARG
    lib.mtb_server_destroy(None)


# ---------------------------------------------------------------- GPU
def _alone(mtb_lib, jobs):
    out = []
    for imgs, L, ref in jobs:
        s = mtb_lib.align_stack(imgs.cuda(), L, 4, ref)
        out.append(s.cpu())
    torch.cuda.synchronize()
    return out


@pytest.mark.gpu
def test_mix_matches_alone_and_oracle(mtb_lib, oracle_mod):
    jobs = _jobs()
    alone = _alone(mtb_lib, jobs)
    biggest = max(mtb_lib.job_bytes(im.shape[0], im.shape[2], im.shape[1], L, 4, ref) for im, L, ref in jobs)
    budget = 3 * biggest  # a few jobs at a time: admission has to wait for memory
    with mtb_lib.Server(budget, slots=4, copy_streams=2) as srv:
        srv.pause()
        ids = [srv.submit(im, L, 4, ref) for im, L, ref in jobs]
        assert all(srv.poll(i) == 1 for i in ids)
        srv.pause(False)
        got = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert st["admitted"] == st["completed"] == len(jobs) and st["failed"] == 0 and st["refused"] == 0
    assert st["bytes_in_use"] == 0 and st["pending"] == 0 and st["running"] == 0
    assert 0 < st["peak_bytes"] <= budget
    assert st["peak_running"] >= 2, "jobs never overlapped"
    for k, ((imgs, L, ref), (shifts, lat, queue)) in enumerate(zip(jobs, got)):
        want = oracle_mod.align_stack(imgs.numpy(), L, 4, ref)["shifts"]
        assert np.array_equal(shifts.numpy(), want), k
        assert torch.equal(shifts, alone[k]), k
        assert lat >= queue >= 0


@pytest.mark.gpu
@pytest.mark.parametrize("copies", [1, 3])
def test_pinned_and_pageable_inputs_agree(mtb_lib, copies):
    """Page-locked inputs are read by the server's copy kernel, pageable ones by
    cudaMemcpyAsync; both give the alone result (sizes with and without a
    ragged last 16 bytes, split over one and three copy streams)."""
    jobs = _jobs()
    alone = _alone(mtb_lib, jobs)
    with mtb_lib.Server(1 << 30, slots=4, copy_streams=copies) as srv:
        ids = []
        for k, (im, L, ref) in enumerate(jobs):
            ids.append((k, srv.submit(im, L, 4, ref)))
            ids.append((k, srv.submit(im.clone(), L, 4, ref)))  # a clone is pageable
        got = [(k, srv.wait(i)[0]) for k, i in ids]
    assert not jobs[0][0].clone().is_pinned()
    for k, g in got:
        assert torch.equal(g, alone[k]), k


@pytest.mark.gpu
def test_arrivals_while_others_run(mtb_lib):
    """Jobs submitted from another thread at random times, with the same stack
    several times in flight at once: every copy gives the alone result."""
    jobs = _jobs()
    alone = _alone(mtb_lib, jobs)
    rng = np.random.default_rng(11)
    order = [int(k) for k in rng.integers(0, len(jobs), 60)]
    gaps = rng.exponential(1 / 2000.0, len(order))
    ids = [None] * len(order)
    with mtb_lib.Server(1 << 30, slots=6, copy_streams=1) as srv:
        def submitter():
            for i, k in enumerate(order):
                time.sleep(gaps[i])
                im, L, ref = jobs[k]
                ids[i] = srv.submit(im, L, 4, ref)

        t = threading.Thread(target=submitter)
        t.start()
        t.join()
        got = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert st["completed"] == len(order) and st["failed"] == 0
    for i, k in enumerate(order):
        assert torch.equal(got[i][0], alone[k]), (i, k)


@pytest.mark.gpu
def test_back_pressure_and_refusals(mtb_lib):
    jobs = _jobs()
    im, L, ref = jobs[0]
    need = mtb_lib.job_bytes(im.shape[0], im.shape[2], im.shape[1], L, 4, ref)
    big, bL, bref = jobs[8]
    with mtb_lib.Server(need + (1 << 20), slots=2, max_pending=2) as srv:
        with pytest.raises(mtb_lib.MtbError) as ei:
            srv.submit(big, bL, 4, bref)  # larger than the whole budget
        assert ei.value.status == mtb_lib.MTB_ERR_BUSY
        with pytest.raises(mtb_lib.MtbError) as ei:
            srv.submit(im, L, 4, im.shape[0])  # ref out of range
        assert ei.value.status == mtb_lib.MTB_ERR_INVALID_ARG
        srv.pause()
        a = srv.submit(im, L, 4, ref)
        b = srv.submit(im, L, 4, ref)
        with pytest.raises(mtb_lib.MtbError) as ei:
            srv.submit(im, L, 4, ref)  # queue full
        assert ei.value.status == mtb_lib.MTB_ERR_BUSY
        st = srv.stats()
        assert st["pending"] == 2 and st["admitted"] == 0 and st["refused"] == 2
        srv.pause(False)
        sa, sb = srv.wait(a)[0], srv.wait(b)[0]
        assert srv.stats()["peak_running"] == 1  # the budget holds one job at a time
        assert srv.poll(a) == mtb_lib.MTB_ERR_INVALID_ARG  # forgotten after wait
    alone = _alone(mtb_lib, [jobs[0]])[0]
    assert torch.equal(sa, alone) and torch.equal(sb, alone)


@pytest.mark.parametrize("bad", ["short", "int64", "strided"])
def test_submit_rejects_bad_out_on_host(bad):
    """The completion callback writes n x 2 int32 into `out`: anything else is
    refused before the job reaches the library (no server or GPU needed)."""
    import paper_2007_06483_gb300 as mtb

    srv = mtb.Server.__new__(mtb.Server)  # checks run before any library call
    srv._h = None
    srv._jobs = {}
    images = torch.zeros((3, 8, 16, 3), dtype=torch.uint8)
    out = {"short": torch.empty((2, 2), dtype=torch.int32),
           "int64": torch.empty((3, 2), dtype=torch.int64),
           "strided": torch.empty((3, 4), dtype=torch.int32)[:, ::2]}[bad]
    with pytest.raises(ValueError, match="out must be"):
        srv.submit(images, 3, out=out)
