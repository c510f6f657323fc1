"""Batches: many stacks of uneven size and exposure count in one persistent,
graph-captured launch; every stack must match the plain path and the oracle
bit for bit, before and after the autotuner changes the tile shapes."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2007_06483_gb300 import synth

# (w, h, n, levels, ref): odd widths, deep levels, windowed coarse levels of
# every radius, level 0 as a window level, several exposures
MIX = [
    (37, 23, 2, 3, 1), (100, 75, 3, 5, 2), (257, 33, 2, 6, 0), (513, 97, 4, 7, 1), (640, 480, 2, 6, 0),
    (600, 450, 4, 8, 2), (1000, 700, 3, 5, 1), (1001, 333, 5, 4, 3), (800, 600, 6, 7, 3), (2, 2, 2, 2, 1),
    (1024, 1024, 2, 11, 0), (333, 222, 3, 5, 1),
]


def _stacks(device="cuda"):
    out = []
    for j, (w, h, n, L, ref) in enumerate(MIX):
        spec = synth.small_spec(300 + j, w, h, n=n, levels=L, shift_range=min(6, (1 << L) - 1), ref=ref)
        out.append({"images": synth.make_stack(spec, device), "levels": L, "noise_tol": 4, "ref_idx": ref})
    return out


def test_batch_rejects_invalid_stack_on_host(mtb_lib):
    bad = mtb_lib.StackDesc(1 << 20, 2, 64, 64, 8, 4, 0, 1 << 20, None, None)  # 64 >> 7 == 0
    arr = (mtb_lib.StackDesc * 1)(bad)
    assert mtb_lib.lib().mtb_batch_workspace_bytes(ctypes.cast(arr, ctypes.c_void_p), 1) == 0
    h = ctypes.c_void_p()
    rc = mtb_lib.lib().mtb_batch_create(ctypes.cast(arr, ctypes.c_void_p), 1, None, 0, ctypes.byref(h))
    assert rc == mtb_lib.MTB_ERR_INVALID_ARG and not h.value
    assert mtb_lib.lib().mtb_batch_create(None, 1, None, 0, ctypes.byref(h)) == mtb_lib.MTB_ERR_INVALID_ARG


@pytest.mark.gpu
def test_batch_matches_plain_path_and_oracle(mtb_lib, oracle_mod):
    stacks = _stacks()
    batch = mtb_lib.Batch(stacks)
    assert batch.config()["graph"]
    for attempt in range(2):
        for k in range(len(stacks)):  # stale outputs must be overwritten
            batch.shifts[k].fill_(-77)
            batch.level_errs[k].fill_(-77)
        batch.run()
        torch.cuda.synchronize()
        assert batch.status() == mtb_lib.MTB_OK
        for k, st in enumerate(stacks):
            L, ref = st["levels"], st["ref_idx"]
            want = oracle_mod.align_stack(st["images"].cpu().numpy(), L, 4, ref)
            assert np.array_equal(batch.shifts[k].cpu().numpy(), want["shifts"]), (k, attempt)
            assert np.array_equal(batch.level_errs[k].cpu().numpy().view(np.uint32), want["level_errs"]), k
            assert np.array_equal(batch.level_shifts[k].cpu().numpy(), want["level_shifts"]), k
            ps, pe, pl = mtb_lib.align_stack(st["images"], L, 4, ref, level_outputs=True)
            assert torch.equal(ps, batch.shifts[k]) and torch.equal(pe, batch.level_errs[k])
    batch.close()


@pytest.mark.gpu
def test_batch_autotuner_keeps_results(mtb_lib):
    stacks = _stacks()
    batch = mtb_lib.Batch(stacks, level_outputs=False)
    batch.run()
    torch.cuda.synchronize()
    before = [s.clone() for s in batch.shifts]
    batch.tune(reps=2)
    cfg = batch.config()
    assert cfg["pyr_runs_per_cta"] in (1, 2, 4) and cfg["bit_chunk_words"] in (512, 1024, 2048, 4096)
    assert cfg["search_waves"] in (1, 2, 4) and cfg["window_kwords"] in (0, 256, 2048)
    for s in batch.shifts:
        s.fill_(-1)
    batch.run()
    torch.cuda.synchronize()
    for a, b in zip(before, batch.shifts):
        assert torch.equal(a, b)
    batch.close()


def test_batch_set_config_rejects_invalid_arguments_on_host(mtb_lib):
    v = (ctypes.c_int * 5)(1, 1024, 1, 0, 2048)
    assert mtb_lib.lib().mtb_batch_set_config(None, v, 5) == mtb_lib.MTB_ERR_INVALID_ARG
    assert mtb_lib.lib().mtb_batch_config(None, v, 5) == mtb_lib.MTB_ERR_INVALID_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("cfg", [(1, 1024, 1, 0), (2, 512, 4, 256), (4, 4096, 2, 2048), (1, 2048, 1, 0)])
def test_batch_every_setting_matches_plain_path(mtb_lib, cfg):
    """The coarse-window budget moves levels between brute-force windows and
    9-candidate hops (0: none windowed); the other settings change item sizes.
    Every setting must give the plain path's shifts, errors and level shifts."""
    stacks = _stacks()
    batch = mtb_lib.Batch(stacks)
    batch.set_config(*cfg)
    got = batch.config()
    assert (got["pyr_runs_per_cta"], got["bit_chunk_words"], got["search_waves"], got["window_kwords"]) == cfg
    assert got["graph"]
    for attempt in range(2):
        batch.run()
        torch.cuda.synchronize()
        assert batch.status() == mtb_lib.MTB_OK
        for k, st in enumerate(stacks):
            ps, pe, pl = mtb_lib.align_stack(st["images"], st["levels"], 4, st["ref_idx"], level_outputs=True)
            assert torch.equal(ps, batch.shifts[k]), (cfg, k)
            assert torch.equal(pe, batch.level_errs[k]), (cfg, k)
            assert torch.equal(pl, batch.level_shifts[k]), (cfg, k)
    with pytest.raises(mtb_lib.MtbError):
        batch.set_config(1, 1024, 1, 100)  # not one of the candidates
    with pytest.raises(mtb_lib.MtbError):
        batch.set_config(3, 1024, 1, 0)
    assert batch.config() == got
    batch.close()


@pytest.mark.gpu
def test_batch_caller_workspace(mtb_lib):
    stacks = _stacks()[:4]
    nbytes = mtb_lib.Batch.workspace_bytes(stacks)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    batch = mtb_lib.Batch(stacks, level_outputs=False, workspace=ws)
    batch.run()
    torch.cuda.synchronize()
    for k, st in enumerate(stacks):
        want = mtb_lib.align_stack(st["images"], st["levels"], 4, st["ref_idx"])
        assert torch.equal(want, batch.shifts[k])
    batch.close()
