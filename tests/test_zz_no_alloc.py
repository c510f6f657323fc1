"""mtb_align_stack_noalloc, the entry point for callers that cannot allocate
device memory while they align (a per-frame loop with a deadline, a plug-in
whose host owns every allocation, a fixed memory budget).  It must give exactly
what mtb_align_stack_ex gives, call after call, although every call reuses the
same fixed scratch array.  This file sorts last so that a run stopping at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2007_06483_gb300 import synth

pytestmark = pytest.mark.gpu

NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024


def _c_entry(mtb):
    lib = ctypes.CDLL(mtb.library_path())
    fn = lib.mtb_align_stack_noalloc
    P, I = ctypes.c_void_p, ctypes.c_int
    fn.restype = I
    fn.argtypes = [P, I, I, I, I, I, I, P, P, P, P]
    return fn


def test_noalloc_matches_align_stack_ex_twice_in_a_row(mtb_lib):
    fn = _c_entry(mtb_lib)
    stream = torch.cuda.current_stream().cuda_stream
    # two different stacks back to back: the second must not see the first's leftovers
    specs = [synth.small_spec(41, 1280, 720, n=4, levels=6, shift_range=40, ref=1), synth.PAIR_640]
    for spec in specs:
        imgs = synth.make_stack(spec, "cuda")
        n = spec.n
        assert mtb_lib.workspace_bytes(n, spec.w, spec.h, spec.levels) <= NOALLOC_SCRATCH_BYTES
        want_s, want_e, want_l = mtb_lib.align_stack(imgs, spec.levels, spec.noise_tol, spec.ref,
                                                     level_outputs=True)
        got_s = torch.full((n, 2), -7, dtype=torch.int32, device="cuda")
        got_e = torch.full((n, spec.levels, 9), -7, dtype=torch.int32, device="cuda")
        got_l = torch.full((n, spec.levels, 2), -7, dtype=torch.int32, device="cuda")
        rc = fn(imgs.data_ptr(), n, spec.w, spec.h, spec.levels, spec.noise_tol, spec.ref, got_s.data_ptr(),
                got_e.data_ptr(), got_l.data_ptr(), stream)
        assert rc == 0, mtb_lib.status_string(rc)
        torch.cuda.synchronize()
        assert torch.equal(got_s, want_s)
        assert torch.equal(got_e, want_e)
        assert torch.equal(got_l, want_l)
        assert np.array_equal(got_s.cpu().numpy(), synth.expected_shifts(spec))


def test_noalloc_rejects_stacks_beyond_its_scratch(mtb_lib):
    fn = _c_entry(mtb_lib)
    imgs = torch.zeros((2, 16, 16, 3), dtype=torch.uint8, device="cuda")
    out = torch.zeros((2, 2), dtype=torch.int32, device="cuda")
    w, h = 6000, 4000  # 2 x 24 MP needs far more than the fixed array
    assert mtb_lib.workspace_bytes(2, w, h, 8) > NOALLOC_SCRATCH_BYTES
    rc = fn(imgs.data_ptr(), 2, w, h, 8, 4, 0, out.data_ptr(), None, None, None)
    assert rc == mtb_lib.MTB_ERR_INVALID_ARG
